// hsb_persist.cu -- persistent tcgen05 kernel running the whole heated
// discrete SB step loop (HdSB, couplings in {-1, 0, +1}) on sm_103a.
//
// Kanao & Goto, arXiv 2203.08361: force Eq. (eq_fd); update Methods Eqs.
// (eq_SyEuY), (eq_SyEuX), (eq_WallX), (eq_WallY), (eq_EuHeat); energy Eq.
// (eq_Ising) evaluated every `eval_every` steps and at the end (K2000 study).
//
// Each CTA owns one tile of 128 spins x 128 replicas for the whole run.  The
// force is formed transposed, F^T = S^T J (the MMA's M dimension is the
// tile's replicas, N its spins), so the tile's positions x and momenta y stay
// in tensor memory next to the FP32 accumulator with lane = replica and
// column = spin (columns 0-127 accumulator, 128-255 x, 256-383 y, FP4 block
// scales at 384), and an epilogue thread owns 32 consecutive spins of one
// replica.  A step moves only J and the sign operand S = sgn(x) through L2.
// One step of a tile is a dependency chain (the force needs the sign tiles
// of every row block), so the roles are arranged to shorten it:
//   warp 0      poller: reads the per-tile "published" flags of the step's
//               operand (one flag per 128-spin chunk, all lanes at once) and
//               raises the pass counter of each load unit (the 128-spin K
//               chunks of two 128-byte slices: two in FP8, four in FP4) whose
//               chunks are all published;
//   warps 1-2   TMA issuers: load g fills stage g % 3 with the unit's two
//               128-byte K slices of J (128 rows, warp 1) and of S (warp 2),
//               one 3-D box of 128 x 128 x 2 bytes each.  Every
//               tile takes its units in a fixed order starting from its own,
//               so the J slice of a load does not wait for any publication:
//               warp 1 copies it as soon as the stage is free and the first
//               loads of a pass have their J before the signs arrive; warp 2
//               copies the S slice once the unit's counter allows (the FP8
//               and FP4 products are exact integers, so the order of the K
//               slices does not change the force);
//   warp 3      MMA: issues tcgen05.mma (kind::f8f6f4, M = N = 128, K = 32;
//               FP4 kind::mxf4, K = 64) from an elected lane of the converged
//               warp (warp-uniform operands issue faster than from one
//               divergent thread).  With kMmaWarps = 2, load t goes to warp
//               3 + t % 2 and its own
//               accumulator (split K); the partial forces are exact integers,
//               so their binary32 sum is the exact force;
//   warps 4-19  epilogue, four warps per 32-lane quadrant (32 replicas) of
//               tensor memory, one per 32-spin column group, in two phases.
//               Phase 1 computes only x~ (sgn(x') = sgn(x~), the walls keep
//               the sign) and writes each thread's 32 signs straight from
//               registers as one row segment of the other operand buffer (FP8
//               two 16-byte stores, FP4 one), then one thread releases the
//               tile's flag at gpu scope.  Phase 2, while the flags travel,
//               repeats the pinned update in full and stores x' and y' in
//               tensor memory; on evaluation steps it also forms the
//               per-replica partial sums of s_i f_i (in-thread over its 32
//               spins, then over the four column groups) and a snapshot of
//               s = sgn(x(t_k)).  Each warp then releases the accumulator.
// A final pass after the last update evaluates E(t_Ns).  The best evaluation
// per replica is chosen afterwards by select_best_kernel.
//
// With the Nose-Hoover thermostat (kNH; Eqs. eq_NH1, eq_NH) the friction
// factor fl32(-xi_r dt) of each replica replaces the heating factor in phase
// 2.  Phase 2 also forms S_r = sum_i y_i'^2 of the tile's rows exactly (q_i =
// 2^24 y_i rounded, q_i^2 split into 22-bit chunks summed over the warp with
// redux and over the quadrants with shared-memory atomics), writes the tile's
// sums to a three-slot buffer and releases a second flag.  Phase 2 of the next
// pass waits for the row blocks' flags of its replica block, adds their sums
// (exact integers) and advances xi before its update.  Phase 1 needs no xi
// (the friction does not move x~), so the wait stays off the critical path.
// Three slots: a tile writes slot p % 3 in pass p only after every tile of its
// replica block has published pass p - 1's signs, hence finished reading
// slot (p - 3) % 3 in pass p - 2.
//
// All CTAs must be co-resident (cooperative launch).  Every wait is bounded:
// mbarrier, ring and flag waits give up after a wall-clock budget, raise the
// CTA's abort flag and the error word; epilogue warps decide to leave through
// a barrier reduction, so they never wait at a named barrier for a warp that
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
// One load is one 3-D box of two 128-byte K slices of each operand's 128
// rows (32 KB per operand): 256 spins in FP8, 512 packed e2m1 values in FP4.
// Three stages of 64 KB.  (Stages of one slice, twice as many copies, were
// slower for both precisions, also with one issuing lane per stage.)
template <bool FP4>
struct PShape {
    static constexpr int Slices = 2;  // 128-byte K slices per load
    static constexpr int Stages = 3;
    static constexpr int StageA = Slices * kPM * kPK;
    static constexpr int StageB = Slices * kPN * kPK;
    static constexpr int ChunksPerLoad = Slices * (FP4 ? 2 : 1);  // 128-spin chunks
};
constexpr int kPStagesMax = 3;
constexpr int kMaxLoads = 32;  // loads per pass (one flag lane per chunk, nblk <= 32)
constexpr int kIssuers = 2;
constexpr int kMmaWarps = 1;  // 2 splits K over two accumulators
constexpr int kFirstMma = 1 + kIssuers;
constexpr int kFirstEpi = kFirstMma + kMmaWarps;
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kPThreads = 32 * kFirstEpi + kEpiThreads;
constexpr uint32_t kPTmemCols = 512;
constexpr uint32_t kColAcc0 = 0;
constexpr uint32_t kColAcc1 = 128;                 // used when kMmaWarps == 2
constexpr uint32_t kColX = 128 * kMmaWarps;
constexpr uint32_t kColY = kColX + 128;
constexpr uint32_t kColSF = kColY + 128;           // FP4: unit block scales (16 columns)
constexpr uint32_t kIdesc = ptx::idesc_e4m3_f32(kPM, kPN);
constexpr uint32_t kIdesc4 = ptx::idesc_mxf4_e2m1(kPM, kPN);
static_assert(kColSF + 16 <= kPTmemCols, "tensor memory columns");

struct __align__(8) PShared {
    uint64_t full[kPStagesMax];
    uint64_t empty[kPStagesMax];
    uint64_t accfull;     // one arrival per MMA warp
    uint64_t tmem_empty;  // every epilogue warp has read the accumulator(s)
    uint64_t drain;       // one arrival per MMA warp once its MMAs have completed
    uint32_t tmem_base;
    int abort;
    int rdy[kMaxLoads];     // load unit u is published for passes < rdy[u] (poller)
    int copies[kPStagesMax][2];  // uses of each stage copied: [stage][J, S] (drain)
    float red[4][kPN];    // per-quadrant energy partials
    // Nose-Hoover (kNH): xi of the tile's replicas, the friction factor of
    // the current pass, and 22-bit chunk sums of q^2 over the tile's rows
    double xi[kPN];
    float gnh[kPN];
    unsigned nhacc[3][kPN];
    // per-step trace: per-quadrant sums of s_i f_i and y_i^2 (traced passes)
    int tre[4][kPN];
    float trt[4][kPN];
};

template <bool FP4>
constexpr size_t persist_smem()
{
    return 1024 + (size_t)PShape<FP4>::Stages * (PShape<FP4>::StageA + PShape<FP4>::StageB) +
           sizeof(PShared);
}
static_assert(persist_smem<false>() <= 232448, "shared memory per CTA is limited to 227 KB");
static_assert(persist_smem<true>() <= 232448, "shared memory per CTA is limited to 227 KB");
static_assert(kPThreads <= 1024, "too many threads per CTA");

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

// The same OR-barrier over the first four epilogue warps (Nose-Hoover xi).
__device__ __forceinline__ bool nh_bar_or(bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred)
        : "memory");
    return r != 0;
}

// Bounded wait by every lane of a warp; false in all lanes if any gave up.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, int *abort, int *err)
{
    const bool ok = ptx::mbar_wait(bar, parity, abort, err);
    return __all_sync(0xFFFFFFFFu, ok);
}

// tcgen05.mma (both operands in shared memory) issued by one elected lane of
// a converged warp; the operand values are warp-uniform.
__device__ __forceinline__ void mma_fp8_elect(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                              uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %3, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %4, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(accumulate), "r"(kIdesc)
        : "memory");
}

// tcgen05.commit from one elected lane: arrives on `bar` when the MMAs this
// lane issued have completed.
__device__ __forceinline__ void commit_elect(uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
            ptx::smem_u32(bar))
        : "memory");
}

// Force of 16 replica columns from tensor memory: the accumulator, plus the
// second one when K is split over two MMA warps (partial forces over
// disjoint K ranges are exact integers, added 8 columns at a time).
__device__ __forceinline__ void load_force(uint32_t tcol, bool two_acc, uint32_t (&f)[16])
{
    ptx::tmem_ld16(tcol + kColAcc0, f);
    if (two_acc) {
#pragma unroll
        for (int p8 = 0; p8 < 2; ++p8) {
            uint32_t f1[8];
            ptx::tmem_ld8(tcol + kColAcc1 + p8 * 8, f1);
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

// q^2 for q = round(2^24 y) (exact scaling, round to nearest even), |y| < 256
// (else *bad), split into 22-bit chunks added to s0, s1, s2; over the 32
// spins of a thread each chunk sum stays below 2^27, over a tile's 128 spins
// below 2^29.
__device__ __forceinline__ void nh_square_chunks(float y, unsigned &s0, unsigned &s1,
                                                 unsigned &s2, bool &bad)
{
    const float s = fabsf(y * 16777216.0f);
    uint64_t v = 0;
    if (s < 4294967296.0f) {
        const uint32_t m = __float2uint_rn(s);  // |round(2^24 y)|, ties to even
        v = (uint64_t)m * m;
    } else {
        bad = true;  // also NaN
    }
    s0 += (unsigned)(v & 0x3FFFFFu);
    s1 += (unsigned)((v >> 22) & 0x3FFFFFu);
    s2 += (unsigned)(v >> 44);
}

// (hi 2^64 + lo) 2^-48 rounded once to binary64 (see nh_update_kernel).
__device__ __forceinline__ double nh_u128_q48_to_double(uint64_t hi, uint64_t lo)
{
    if (hi == 0)
        return __dmul_rn(__ull2double_rn(lo), 0x1p-48);
    const int lz = __clzll((long long)hi);
    uint64_t t = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
    if (lo << lz)
        t |= 1ull;
    return __dmul_rn(__ull2double_rn(t),
                     __longlong_as_double((long long)(1023 + 16 - lz) << 52));
}

}  // namespace

// The step loop of one tile.  kFP4: J and S in packed e2m1 (rows of Kp/2
// bytes), kind::mxf4 MMAs with unit block scales, the sign tile published as
// nibbles; otherwise FP8 e4m3 and kind::f8f6f4.
template <bool kNH, bool kFP4>
__device__ __forceinline__ void persistent_body(const CUtensorMap *tmapA,
                                                const CUtensorMap *tmapB0,
                                                const CUtensorMap *tmapB1, const PersistArgs &a)
{
    constexpr int kPStages = PShape<kFP4>::Stages;
    constexpr int kPStageA = PShape<kFP4>::StageA;
    constexpr int kPStageB = PShape<kFP4>::StageB;
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
    // loads of a pass: unit u covers K chunks kCpl u .. kCpl u + kCpl - 1; a
    // chunk past the end reads as zero.  Every tile takes the units in the order u0, u0 + 1,
    // ... cyclically from its own (the first published, by this CTA), so
    // tiles sharing rows ask for different lines at a time
    constexpr int kCpl = PShape<kFP4>::ChunksPerLoad;
    const int nload = (nblk + kCpl - 1) / kCpl;
    const int u0 = mb / kCpl;
    const int passes = a.nsteps + a.final_pass;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPStages; ++s) {
            ptx::mbar_init(&sh->full[s], 1);
            ptx::mbar_init(&sh->empty[s], 1);
        }
        ptx::mbar_init(&sh->accfull, kMmaWarps);
        ptx::mbar_init(&sh->tmem_empty, kEpiWarps);
        ptx::mbar_init(&sh->drain, kMmaWarps);
        for (int s = 0; s < kPStages; ++s)
            sh->copies[s][0] = sh->copies[s][1] = 0;
        for (int u = 0; u < kMaxLoads; ++u)
            sh->rdy[u] = 0;
        sh->abort = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 1 && lane == 0) {
        ptx::prefetch_tmap(tmapA);
        ptx::prefetch_tmap(tmapB0);
        ptx::prefetch_tmap(tmapB1);
    }
    if (warp == kFirstMma)
        ptx::tmem_alloc(&sh->tmem_base, kPTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    if (kFP4) {
        // unit block scales (UE8M0 0x7F = 2^0) in 16 columns of every lane,
        // before the first MMA reads them
        if (warp >= kFirstEpi && warp < kFirstEpi + 4) {
            uint32_t one[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                one[j] = 0x7F7F7F7Fu;
            ptx::tmem_st16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + kColSF, one);
            ptx::tmem_st_wait();
        }
        ptx::tc_fence_before();
        __syncthreads();
        ptx::tc_fence_after();
    }

    if (warp == 0) {
        // ------------------------------------------------------------ poller
        // lane c reads the flag of chunk c (tile (c, rb)) for each pass; once
        // every chunk of a load unit is published, lane u raises the unit's
        // pass counter, which the S issuer waits on
        bool fail = false;
        const uint32_t all_units = nload >= 32 ? 0xFFFFFFFFu : ((1u << nload) - 1u);
        for (int kl = 0; kl < passes && !fail; ++kl) {
            uint32_t pending = nblk >= 32 ? 0xFFFFFFFFu : ((1u << nblk) - 1u);
            uint32_t have = 0;
            uint32_t left = all_units;
            const unsigned long long t0 = ptx::globaltimer();
            int idle = 0;
            while (left) {
                bool ready = false;
                if (lane < nblk && ((pending >> lane) & 1u))
                    ready = ptx::ld_acquire_gpu(&a.flags[flag_index(lane, rb, a.nrb)]) >= kl;
                const uint32_t rmask = __ballot_sync(0xFFFFFFFFu, ready);
                have |= rmask;
                pending &= ~rmask;
                bool unit = false;
                if ((left >> lane) & 1u) {
                    const int c0 = kCpl * lane;
                    const int nc = nblk - c0 < kCpl ? nblk - c0 : kCpl;
                    const uint32_t need = ((1u << nc) - 1u) << c0;
                    unit = (have & need) == need;
                }
                if (unit)
                    ptx::st_release_cta_shared(&sh->rdy[lane], kl + 1);
                const uint32_t umask = __ballot_sync(0xFFFFFFFFu, unit);
                left &= ~umask;
                if (!umask && left) {
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
    } else if (warp <= kIssuers) {
        // ------------------------------------------------------- TMA issuers
        // Both issuers serve every load g in order (stage g % kPStages).  Warp
        // 1 copies the J slice as soon as the stage is free (J does not wait
        // for the step's signs, so a pass's first loads have their J before
        // its signs are published) and posts the stage's expected bytes (its
        // one arrival); warp 2 copies the S slice once the unit is published.
        // A copy of S that lands first takes the transaction count below zero
        // until then: it cannot belong to the previous use, whose MMAs had
        // completed before the stage was free.
        if (lane == 0) {
            const bool jl = warp == 1;
            const int total = passes * nload;
            int used = 0;
            for (int g = 0; g < total; ++g) {
                const int kl = g / nload;
                int u = u0 + (g - kl * nload);
                if (u >= nload)
                    u -= nload;
                const int s = g % kPStages;
                const uint32_t ph = (uint32_t)(g / kPStages) & 1u;
                if (!ptx::mbar_wait(&sh->empty[s], ph ^ 1u, &sh->abort, a.err))
                    break;
                if (jl) {
                    ptx::mbar_expect_tx(&sh->full[s], (uint32_t)(kPStageA + kPStageB));
                    ptx::tma_load_3d(sA + (size_t)s * kPStageA, tmapA, 0, m0,
                                     PShape<kFP4>::Slices * u, &sh->full[s]);
                } else {
                    if (!ptx::wait_count(&sh->rdy[u], kl + 1, &sh->abort, a.err))
                        break;
                    ptx::fence_proxy_async_global();
                    const CUtensorMap *mapB = ((a.par0 + kl) & 1) ? tmapB1 : tmapB0;
                    ptx::tma_load_3d(sB + (size_t)s * kPStageB, mapB, 0, r0,
                                     PShape<kFP4>::Slices * u, &sh->full[s]);
                }
                used = g + 1;
            }
            // the uses of each stage this thread copied, for the drain
            for (int s = 0; s < kPStages; ++s)
                sh->copies[s][jl ? 0 : 1] = used > s ? (used - 1 - s) / kPStages + 1 : 0;
        }
    } else if (warp < kFirstEpi) {
        // --------------------------------------------------------------- MMA
        // descriptors of stage 0; a stage or K step further is a plain add on
        // the 14-bit start-address field (addresses < 256 KB)
        const int mw = warp - kFirstMma;
        const uint32_t dcol = tmem + (mw ? kColAcc1 : kColAcc0);
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
            for (int t = mw; t < nload; t += kMmaWarps) {
                const int g = kl * nload + t;
                const int s = g % kPStages;
                const uint32_t ph = (uint32_t)(g / kPStages) & 1u;
                if (!warp_wait(&sh->full[s], ph, &sh->abort, a.err)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint64_t ad = adesc0 + (uint64_t)((s * kPStageA) >> 4);
                const uint64_t bd = bdesc0 + (uint64_t)((s * kPStageB) >> 4);
                // each 128-byte K slice of the operand rows: four MMAs of 32
                // bytes (K = 32 e4m3 or K = 64 e2m1 values)
#pragma unroll
                for (int c = 0; c < PShape<kFP4>::Slices; ++c) {
#pragma unroll
                    for (int kk = 0; kk < kPK / 32; ++kk) {
                        // A = the S slice (replicas), B = the J slice (spins):
                        // the accumulator holds F^T, lane = replica
                        const uint64_t sk = bd + (uint64_t)((c * kPN * kPK + kk * 32) >> 4);
                        const uint64_t jk = ad + (uint64_t)((c * kPM * kPK + kk * 32) >> 4);
                        const uint32_t acc = (mine | c | kk) != 0 ? 1u : 0u;
                        if (kFP4)
                            ptx::mma_mxf4_elect(dcol, sk, jk, kIdesc4, tmem + kColSF,
                                                tmem + kColSF, acc);
                        else
                            mma_fp8_elect(dcol, sk, jk, acc);
                    }
                }
                commit_elect(&sh->empty[s]);
                ++mine;
            }
            if (!ok)
                break;
            if (mine > 0)
                commit_elect(&sh->accfull);
            else if (lane == 0)
                ptx::mbar_arrive(&sh->accfull);  // no pair of this pass for this warp
        }
        commit_elect(&sh->drain);  // arrives once this warp's MMAs have completed
    } else {
        // ---------------------------------------------------------- epilogue
        // The force is formed transposed (lane = replica, column = spin), so
        // a thread owns 32 consecutive spins of one replica: its signs are
        // one contiguous row segment of the next operand, stored straight
        // from registers.
        const int ew = warp - kFirstEpi;    // 0..15
        const int q = warp & 3;             // tensor-memory lane quadrant
        const int cg = ew >> 2;             // spin column group (32 spins)
        const int et = threadIdx.x - 32 * kFirstEpi;  // 0..511
        const int rl = q * 32 + lane;       // replica of this thread within the tile
        const int r = r0 + rl;
        const int ib = m0 + cg * 32;        // first of this thread's 32 spins
        const uint32_t col0 = (uint32_t)(cg * 32);
        const bool two_acc = kMmaWarps > 1 && nload > 1;  // a second accumulator has loads
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const size_t plane = (size_t)a.Rp * a.Np;
        // live spins of this thread's 32 (padded spins publish a zero code)
        const uint32_t live = ib + 32 <= a.N ? 0xFFFFFFFFu
                              : ib >= a.N   ? 0u
                                            : ((1u << (a.N - ib)) - 1u);
        uint8_t *const srow_a = a.S8a + (kFP4 ? (size_t)r * (a.Kp / 2) + ib / 2
                                              : (size_t)r * a.Np + ib);
        uint8_t *const srow_b = a.S8b + (kFP4 ? (size_t)r * (a.Kp / 2) + ib / 2
                                              : (size_t)r * a.Np + ib);

        // initial state of the tile into tensor memory
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t xr[16], yr[16];
            const float4 *xs = reinterpret_cast<const float4 *>(a.X + (size_t)r * a.Np + ib + 16 * h);
            const float4 *ys = reinterpret_cast<const float4 *>(a.Y + (size_t)r * a.Np + ib + 16 * h);
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
            ptx::tmem_st16(tmem + lane_off + kColX + col0 + 16 * h, xr);
            ptx::tmem_st16(tmem + lane_off + kColY + col0 + 16 * h, yr);
        }
        ptx::tmem_st_wait();
        if (kNH && et < kPN) {
            // xi(t_k_begin) of this tile's replicas and its friction factor;
            // the epilogue barrier of the first pass orders these stores
            const double x0 = a.xi[r0 + et];
            sh->xi[et] = x0;
            sh->gnh[et] = __double2float_rn(__dmul_rn(-x0, a.dt64));
            sh->nhacc[0][et] = sh->nhacc[1][et] = sh->nhacc[2][et] = 0u;
        }
        bool nh_bad = false;

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
            // traced time t_k (per-step trace): energy and T_inst of the state
            // before this pass's update
            const int tm = (!final_pass && a.trace_every > 0 && k % a.trace_every == 0)
                               ? k / a.trace_every
                               : -1;
            const float pk = final_pass ? 0.f : pk_next;
            const uint64_t pk2 = f2_pack(pk, pk);
            if (kl + 1 < a.nsteps)
                pk_next = a.pk[k + 1];  // p_k of the next pass, off the critical path

            // Nose-Hoover: xi_k = xi_{k-1} + (dt/M)(S - N T), S = sum_i
            // y_i(t_k)^2 from every row block's sums of the previous pass (Eq.
            // eq_NH).  Warps 0-3 (one thread per replica column) do it while
            // the MMA runs; phase 2 reads the factor after the phase-1 barrier.
            bool ok_nh = true;
            if (kNH && kl > 0 && ew < 4) {
                if (ew == 0) {
                    bool mine = lane >= nblk;
                    const unsigned long long t0 = ptx::globaltimer();
                    int idle = 0;
                    while (!__all_sync(0xFFFFFFFFu, mine)) {
                        if (!mine)
                            mine = ptx::ld_acquire_gpu(
                                       &a.nhflags[flag_index(lane, rb, a.nrb)]) >= kl;
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
                            ok_nh = false;
                            break;
                        }
                    }
                }
                ok_nh = !nh_bar_or(!ok_nh);
                if (ok_nh) {
                    const unsigned long long *src =
                        a.nhpart + ((size_t)((kl - 1) % 3) * nblk * a.Rp + r0 + et) * 2;
                    // eight row blocks' sums in flight at a time (one L2 round
                    // trip per eight, not per block)
                    uint64_t hi = 0, lo = 0;
                    for (int b0 = 0; b0 < nblk; b0 += 8) {
                        uint64_t bh[8], bl[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const bool in = b0 + u < nblk;
                            const unsigned long long *pb = src + (size_t)(b0 + u) * a.Rp * 2;
                            bh[u] = in ? __ldcg(pb) : 0ull;
                            bl[u] = in ? __ldcg(pb + 1) : 0ull;
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const uint64_t l = lo + bl[u];
                            hi += bh[u] + (l < lo ? 1ull : 0ull);
                            lo = l;
                        }
                    }
                    const double S = nh_u128_q48_to_double(hi, lo);
                    const double x =
                        __dadd_rn(sh->xi[et], __dmul_rn(a.nh_h, __dsub_rn(S, a.nh_NT)));
                    sh->xi[et] = x;
                    sh->gnh[et] = __double2float_rn(__dmul_rn(-x, a.dt64));
                }
            }
            // x and y of the first 16 spins (the MMA does not write them) and
            // v = p_k x of their update, formed in the MMA's shadow
            uint32_t xpre[16], ypre[16];
            uint64_t vpre[8];
            ptx::tmem_ld16(tmem + lane_off + kColX + col0, xpre);
            ptx::tmem_ld16(tmem + lane_off + kColY + col0, ypre);
            ptx::tmem_ld_wait(xpre);
            ptx::tmem_ld_wait(ypre);
#pragma unroll
            for (int j = 0; j < 16; j += 2)
                vpre[j / 2] = f2_fma(pk2, f2_pack_bits(xpre[j], xpre[j + 1]), k2.z);
            // one warp waits for the accumulator; the others block at the
            // barrier after it, leaving the schedulers to the poller, the
            // issuers and the MMA warp while the force is formed
            const bool ok =
                (ew != 0 || ptx::mbar_wait(&sh->accfull, (uint32_t)kl & 1u, &sh->abort, a.err)) &&
                ok_nh;
            if (epi_bar_or(!ok)) {
                left = true;
                break;
            }
            ptx::tc_fence_after();

            if (!final_pass) {
                // ---- phase 1: only sgn(x') = sgn(x~) of this thread's 32
                // spins, published before the rest of the update (the next
                // step of every tile waits for it).  The operations are those
                // of the update up to p = q yt; x~ = fl(x + p) is negative
                // exactly when p < -x (a nonzero sum of two binary32 values
                // does not round to zero, a zero sum rounds to +0).  FP8: one
                // sign byte per spin (+1 = 0x38, -1 = 0xB8), two 16-byte
                // stores; FP4: one e2m1 code per spin, spins 2m and 2m + 1 in
                // the low and high nibble of a byte, one 16-byte store.
                uint8_t *dst = ((a.par0 + kl + 1) & 1) ? srow_b : srow_a;
                uint32_t w4[4];  // FP4: the 16 bytes of both halves
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t f[16], xr[16], yr[16];
                    uint64_t v[8];
                    load_force(tmem + lane_off + col0 + 16 * h, two_acc, f);
                    if (h == 0) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            xr[j] = xpre[j];
                            yr[j] = ypre[j];
                        }
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            v[j] = vpre[j];
                    } else {
                        ptx::tmem_ld16(tmem + lane_off + kColX + col0 + 16, xr);
                        ptx::tmem_ld16(tmem + lane_off + kColY + col0 + 16, yr);
                        ptx::tmem_ld_wait(xr);
                        ptx::tmem_ld_wait(yr);
#pragma unroll
                        for (int j = 0; j < 16; j += 2)
                            v[j / 2] = f2_fma(pk2, f2_pack_bits(xr[j], xr[j + 1]), k2.z);
                    }
                    // the negative spins' sign bits placed in their codes:
                    // FP8 bit 7 of byte j (0x38 -> 0xB8), FP4 bit 3 of
                    // nibble j (0x2 -> 0xA); m = all ones when negative
                    uint32_t negw[kFP4 ? 2 : 4] = {};
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const uint64_t u = f2_fma(k2.c0, f2_pack_bits(f[j], f[j + 1]), k2.z);
                        const uint64_t w = f2_sub(u, v[j / 2]);
                        const uint64_t wd = f2_fma(w, k2.dt, k2.z);
                        const uint64_t yt = f2_add(f2_pack_bits(yr[j], yr[j + 1]), wd);
                        const uint64_t qy = f2_fma(k2.q, yt, k2.z);
                        const uint32_t mk0 = 0u - (uint32_t)(f2_lo(qy) < -__uint_as_float(xr[j]));
                        const uint32_t mk1 =
                            0u - (uint32_t)(f2_hi(qy) < -__uint_as_float(xr[j + 1]));
                        if (kFP4) {
                            negw[j / 8] |= (mk0 & (0x8u << (4 * (j % 8)))) |
                                           (mk1 & (0x8u << (4 * ((j + 1) % 8))));
                        } else {
                            negw[j / 4] |= (mk0 & (0x80u << (8 * (j % 4)))) |
                                           (mk1 & (0x80u << (8 * ((j + 1) % 4))));
                        }
                    }
                    const uint32_t lv = (live >> (16 * h)) & 0xFFFFu;
                    if (kFP4) {
#pragma unroll
                        for (int m = 0; m < 2; ++m) {
                            uint32_t wd4 = 0x22222222u | negw[m];
                            if (lv != 0xFFFFu)  // padded spins publish 0
                                wd4 &= nibble_mask8((lv >> (8 * m)) & 0xFFu);
                            w4[2 * h + m] = wd4;
                        }
                    } else {
                        uint32_t wv[4];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            wv[m] = 0x38383838u | negw[m];
                            if (lv != 0xFFFFu)  // padded spins publish 0
                                wv[m] &= byte_mask4((lv >> (4 * m)) & 0xFu);
                        }
                        *reinterpret_cast<uint4 *>(dst + 16 * h) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                    }
                }
                if (kFP4)
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                epi_bar();
                if (et == 0 && !(mb == a.drop_mb && rb == 0)) {
                    // every epilogue thread's S stores precede the barrier; the
                    // gpu-scope release (cumulative) publishes them with the flag
                    ptx::fence_proxy_async_global();
                    ptx::st_release_gpu(&a.flags[flag_index(mb, rb, a.nrb)], kl + 1);
                }
            }

            // ---- phase 2: energy of s(t_k) on evaluation passes, the trace
            // sums on traced passes, and the full update of x and y in tensor
            // memory (off the critical path: the next force needs the flags of
            // every tile first)
            float gfr = 0.f;  // Nose-Hoover friction factor of this replica
            if (kNH)
                gfr = sh->gnh[rl];
            int esum = 0;     // sum of s_i f_i over this thread's spins (exact)
            float ysum = 0.f; // sum of y_i(t_k)^2 over them (trace)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t f[16], xr[16], yr[16];
                ptx::tmem_ld16(tmem + lane_off + kColX + col0 + 16 * h, xr);
                ptx::tmem_ld16(tmem + lane_off + kColY + col0 + 16 * h, yr);
                load_force(tmem + lane_off + col0 + 16 * h, two_acc, f);
                ptx::tmem_ld_wait(xr);
                ptx::tmem_ld_wait(yr);
                if (e >= 0 || tm >= 0) {
                    uint32_t sb[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const bool lv = (live >> (16 * h + j)) & 1u;
                        const float x0 = __uint_as_float(xr[j]);
                        const int fj = (int)__uint_as_float(f[j]);  // exact integer force
                        esum += lv ? (x0 >= 0.f ? fj : -fj) : 0;
                        if (tm >= 0) {
                            const float y0 = __uint_as_float(yr[j]);
                            ysum = __fadd_rn(ysum, __fmul_rn(y0, y0));  // y_i(t_k)^2 (Eq. eq_TInst)
                        }
                        sb[j >> 2] |= (lv ? (uint32_t)fp8_sign(x0) : 0u) << (8 * (j & 3));
                    }
                    if (e >= 0)
                        *reinterpret_cast<uint4 *>(a.Snap + (size_t)e * plane + (size_t)r * a.Np +
                                                   ib + 16 * h) =
                            make_uint4(sb[0], sb[1], sb[2], sb[3]);
                }
                if (!final_pass) {
                    StepConsts2 kn = k2;
                    if (kNH)
                        kn.g = f2_pack(gfr, gfr);  // per-replica friction in place of gamma dt
                    // two spins per packed binary32 operation
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        float xn0, xn1;
                        uint64_t yn;
                        sb_update2(f2_pack_bits(f[j], f[j + 1]), f2_pack_bits(xr[j], xr[j + 1]),
                                   f2_pack_bits(yr[j], yr[j + 1]), pk2, kn, xn0, xn1, yn);
                        xr[j] = __float_as_uint(xn0);
                        xr[j + 1] = __float_as_uint(xn1);
                        yr[j] = (uint32_t)yn;
                        yr[j + 1] = (uint32_t)(yn >> 32);
                    }
                    ptx::tmem_st16(tmem + lane_off + kColX + col0 + 16 * h, xr);
                    ptx::tmem_st16(tmem + lane_off + kColY + col0 + 16 * h, yr);
                }
            }
            ptx::tc_fence_before();
            if (!final_pass)
                ptx::tmem_st_wait();
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive(&sh->tmem_empty);  // this warp has read the accumulator
            if (e >= 0 || tm >= 0) {
                // the four spin column groups' sums of each replica
                if (e >= 0)
                    sh->red[cg][rl] = (float)esum;
                if (tm >= 0) {
                    sh->tre[cg][rl] = esum;
                    sh->trt[cg][rl] = ysum;
                }
                epi_bar();
                if (et < kPN && e >= 0) {
                    const float s = sh->red[0][et] + sh->red[1][et] + sh->red[2][et] + sh->red[3][et];
                    a.Epart[((size_t)e * nblk + mb) * a.Rp + r0 + et] = s;
                }
                if (et < kPN && tm >= 0) {
                    const size_t o = ((size_t)tm * nblk + mb) * a.Rp + r0 + et;
                    a.trE[o] = (float)(sh->tre[0][et] + sh->tre[1][et] + sh->tre[2][et] +
                                       sh->tre[3][et]);
                    a.trT[o] = sh->trt[0][et] + sh->trt[1][et] + sh->trt[2][et] + sh->trt[3][et];
                }
            }
            if (kNH && !final_pass) {
                // this tile's sums of q^2 of y(t_{k+1}) (in tensor memory; the
                // accumulator is already released): slot kl % 3, then the
                // flag.  Each thread sums the 22-bit chunks of q^2 over its 32
                // spins (each chunk sum below 2^27); one shared-memory atomic
                // per chunk adds them to the replica's sums
                unsigned s0 = 0u, s1 = 0u, s2 = 0u;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t yr[16];
                    ptx::tmem_ld16(tmem + lane_off + kColY + col0 + 16 * h, yr);
                    ptx::tmem_ld_wait(yr);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        nh_square_chunks(__uint_as_float(yr[j]), s0, s1, s2, nh_bad);
                }
                atomicAdd(&sh->nhacc[0][rl], s0);
                atomicAdd(&sh->nhacc[1][rl], s1);
                atomicAdd(&sh->nhacc[2][rl], s2);
                epi_bar();  // every warp's atomics are in
                if (et < kPN) {
                    const uint64_t c0 = sh->nhacc[0][et], c1 = sh->nhacc[1][et],
                                   c2 = sh->nhacc[2][et];
                    sh->nhacc[0][et] = sh->nhacc[1][et] = sh->nhacc[2][et] = 0u;
                    const uint64_t lo0 = c0 + (c1 << 22);
                    const uint64_t lo = lo0 + (c2 << 44);
                    const uint64_t hi = (c2 >> 20) + (lo < lo0 ? 1ull : 0ull);
                    unsigned long long *dst =
                        a.nhpart + ((size_t)(kl % 3) * nblk * a.Rp + (size_t)mb * a.Rp + r0 + et) * 2;
                    dst[0] = hi;
                    dst[1] = lo;
                }
                epi_bar();
                if (et == 0)
                    ptx::st_release_gpu(&a.nhflags[flag_index(mb, rb, a.nrb)], kl + 1);
                if (nh_bad)
                    atomicExch(a.err, kErrRange);
            }
        }
        if (kNH && !left && mb == 0 && et < kPN)
            a.xi[r0 + et] = sh->xi[et];  // xi after the last update (final pass)

        // final state back to global memory
        if (!left) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t xr[16], yr[16];
                ptx::tmem_ld16(tmem + lane_off + kColX + col0 + 16 * h, xr);
                ptx::tmem_ld16(tmem + lane_off + kColY + col0 + 16 * h, yr);
                ptx::tmem_ld_wait();
                float4 *xd = reinterpret_cast<float4 *>(a.X + (size_t)r * a.Np + ib + 16 * h);
                float4 *yd = reinterpret_cast<float4 *>(a.Y + (size_t)r * a.Np + ib + 16 * h);
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

    // drain before tensor memory and shared memory are given up (every exit
    // path): the last copy into each stage has landed and every MMA has
    // completed, each wait bounded.  A stage whose last use was never armed
    // (its arming warp gave up first) waits out the bound, with the error
    // word set.
    // A use whose S slice was never copied (the S issuer gave up first) is
    // completed here with a stand-in for its bytes; a use never armed (only
    // possible when J gave up first) is armed for what was copied.
    __syncthreads();
    if (threadIdx.x < kPStages) {
        const int st = threadIdx.x;
        const int jc = sh->copies[st][0], sc = sh->copies[st][1];
        const int U = jc > sc ? jc : sc;
        if (U > 0) {
            const uint32_t landing = (jc >= U ? kPStageA : 0) + (sc >= U ? kPStageB : 0);
            if (jc >= U) {
                if (landing < (uint32_t)(kPStageA + kPStageB))
                    ptx::mbar_complete_tx(&sh->full[st], (uint32_t)(kPStageA + kPStageB) - landing);
            } else {
                ptx::mbar_expect_tx(&sh->full[st], landing);
            }
            ptx::mbar_drain(&sh->full[st], (uint32_t)(U - 1) & 1u, a.err);
        }
    }
    if (warp >= kFirstMma && warp < kFirstEpi)
        ptx::mbar_drain(&sh->drain, 0u, a.err);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == kFirstMma)
        ptx::tmem_dealloc(tmem, kPTmemCols);
}

template <bool kNH>
__global__ void __launch_bounds__(kPThreads, 1)
tc_fp8_persistent_kernel(const __grid_constant__ CUtensorMap tmapA,
                         const __grid_constant__ CUtensorMap tmapB0,
                         const __grid_constant__ CUtensorMap tmapB1, const PersistArgs a)
{
    persistent_body<kNH, false>(&tmapA, &tmapB0, &tmapB1, a);
}

template <bool kNH>
__global__ void __launch_bounds__(kPThreads, 1)
tc_fp4_persistent_kernel(const __grid_constant__ CUtensorMap tmapA,
                         const __grid_constant__ CUtensorMap tmapB0,
                         const __grid_constant__ CUtensorMap tmapB1, const PersistArgs a)
{
    persistent_body<kNH, true>(&tmapA, &tmapB0, &tmapB1, a);
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

namespace {

template <bool FP4>
bool persistent_fits(int Np, int Rp)
{
    const int nblk = Np / kPM;
    const int nrb = Rp / kPN;
    if (nblk < 1 || nblk > 32 || nrb < 1)
        return false;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    // both instantiations of a precision have the same block size and shared memory
    auto kern = FP4 ? tc_fp4_persistent_kernel<false> : tc_fp8_persistent_kernel<false>;
    const size_t smem = persist_smem<FP4>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, smem) !=
        cudaSuccess)
        return false;
    return (long long)nblk * nrb <= (long long)per_sm * sms;
}

template <bool FP4>
cudaError_t launch_persistent(cudaStream_t st, const CUtensorMap &mA, const CUtensorMap &mB0,
                              const CUtensorMap &mB1, const PersistArgs &a)
{
    auto kern = FP4 ? (a.nh ? tc_fp4_persistent_kernel<true> : tc_fp4_persistent_kernel<false>)
                    : (a.nh ? tc_fp8_persistent_kernel<true> : tc_fp8_persistent_kernel<false>);
    const size_t smem = persist_smem<FP4>();
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nblk, a.nrb, 1);
    cfg.blockDim = dim3(kPThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, mA, mB0, mB1, a);
}

}  // namespace

bool tc_persistent_fits(int Np, int Rp) { return persistent_fits<false>(Np, Rp); }

bool tc_fp4_persistent_fits(int Np, int Rp) { return persistent_fits<true>(Np, Rp); }

cudaError_t launch_tc_fp8_persistent(cudaStream_t st, const TcPlan *plan, const PersistArgs &a)
{
    if (!plan || a.Np != plan->Np || a.Rp > plan->Rp || a.Rp % kPN != 0 || a.nblk > 32)
        return cudaErrorInvalidValue;
    if (a.nh && (!a.xi || !a.nhpart || !a.nhflags || !a.final_pass))
        return cudaErrorInvalidValue;
    return launch_persistent<false>(st, plan->mapA3, plan->mapB3[0], plan->mapB3[1], a);
}

cudaError_t launch_tc_fp4_persistent(cudaStream_t st, const TcPlan *plan, const PersistArgs &a)
{
    if (!plan || a.Np != plan->Np || a.Rp > plan->Rp || a.Rp % kPN != 0 || a.nblk > 32 ||
        a.Kp != plan->Kp || a.Kp < a.Np || a.Kp % 256 != 0)
        return cudaErrorInvalidValue;
    if (a.nh && (!a.xi || !a.nhpart || !a.nhflags || !a.final_pass))
        return cudaErrorInvalidValue;
    return launch_persistent<true>(st, plan->mapA3, plan->mapB3[0], plan->mapB3[1], a);
}

cudaError_t launch_select_best(cudaStream_t st, const float *Epart, const uint8_t *Snap,
                               int n_evals, int nblk, int N, int Np, int R, int Rp,
                               double *Ebest, int8_t *Sbest)
{
    select_best_kernel<<<R, 256, 0, st>>>(Epart, Snap, n_evals, nblk, N, Np, Rp, Ebest, Sbest);
    return cudaGetLastError();
}

}  // namespace hsb
