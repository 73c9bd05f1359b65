// hsb_tc.cu -- one-step tensor-core (tcgen05) kernel of libhsb for sm_103a,
// used when the persistent step loop does not fit (large N, many tiles) and
// on the one-launch-per-step schedule (with the per-step trace and the
// Nose-Hoover friction factor per replica where asked).
//
// Discrete heated SB with couplings in {-1, 0, +1} (HdSB; Kanao & Goto,
// arXiv 2203.08361, Eq. (eq_fd) and Methods): the force F = J sgn(X) of all
// replicas is one GEMM with M = spins, N = replicas, K = spins.  J and sgn(X)
// are FP8 e4m3 (+1 = 0x38, -1 = 0xB8, 0 = 0x00), every product is -1, 0 or +1
// and every partial sum an integer of magnitude < 2^24, so FP32 accumulation
// in tensor memory is exact and the force equals the integer J sgn(x).
//
// A persistent grid, one CTA per SM, walks tiles of 128 spins x 256
// replicas (FP4: 192) band by band: the replica blocks are cut into as few
// bands as keep a band's S rows within an L2 budget, and inside a band the
// replica blocks run fastest, so that the CTAs running at one time share a
// few row blocks of J in L2 (J streams from HBM once per band and step) and
// the band's S rows stay in L2 for all row blocks.  x and y go through L2
// with an evict-first policy.  Per CTA:
//   warps 0-3  TMA issuers: warps 0 and 1 load the J box (128 rows x 128 B)
//              of even and odd K chunks, warps 2 and 3 the S box (256 rows x
//              128 B), into a ring of four 48 KB stages (FP4: 40 KB).
//              Copies from one thread complete one after another, so four
//              issuing threads keep the ring full; every stage is always
//              served by the same two issuers, so their parity waits see each
//              phase in order;
//   warp 4     MMA: tcgen05.mma kind::f8f6f4, M = 128, N = 256, K = 32,
//              issued from an elected lane of the converged warp (a 128 x 256
//              x 32 instruction keeps the tensor core busy even from one warp)
//              into one of two 256-column accumulators, alternating by tile,
//              so the epilogue of a tile overlaps the next tile's force;
//   warps 5-12 epilogue, two warps per 32-lane quadrant (128 replica columns
//              each): the accumulator, x and y of the tile from global memory,
//              the pinned spin update, x' and y' in place, sgn(x') as the next
//              step's FP8 operand; on evaluation steps the per-replica partial
//              sums of s_i f_i, with a trace the sums of y_i(t_k)^2.
// Replica columns past Rp (the last tile of an odd number of 128-replica
// blocks) are computed from whatever the operand rows hold and never stored.
// Every wait is bounded (a wall-clock budget); a wait that gives up sets the
// error word and makes the other roles leave their loops; the epilogue warps
// decide to leave through a barrier reduction, and the CTA frees its tensor
// memory before it exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsb_device.cuh"
#include "hsb_internal.cuh"
#include "hsb_ptx.cuh"
#include "hsb_sched.cuh"

namespace hsb {

namespace {

constexpr int kBM = 128;            // spins per tile (MMA M, tensor-memory lanes)
constexpr int kBN = 256;            // replicas per FP8 tile (MMA N, accumulator columns)
constexpr int kBN4 = 192;           // replicas per FP4 tile: two accumulators and the
                                    // unit block scales fit the 512 tensor-memory columns
constexpr int kBK = 128;            // K bytes per stage (one 128-byte swizzle row)
constexpr int kStageA = kBM * kBK;  // 16 KB
constexpr int kIssuers = 4;
constexpr int kMmaWarp = kIssuers;
constexpr int kFirstEpi = kMmaWarp + 1;
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 32 * kFirstEpi + kEpiThreads;
constexpr uint32_t kTmemCols = 512;  // two accumulators (+ the FP4 block scales)
// S rows of one replica band: the band stays in L2 while J and x, y stream
// past it (data read by SMs of both dies may be held in both halves of L2)
constexpr size_t kSBandBytes = (size_t)40 << 20;
constexpr bool kRotateK = true;
// From this padded size on, one step runs on CTA pairs (tc_step_pair_kernel).
constexpr int kPairMinNp = 1024;

// FP8: kind::f8f6f4 e4m3, K = 32 per instruction.  FP4: kind::mxf4 with packed
// e2m1 operands (+1 = 0x2, -1 = 0xA, 0 = 0x0, element 2j in the low nibble of
// byte j), K = 64 per instruction, block scales UE8M0 1.0 read from tensor
// memory; both take 32 bytes of each operand row per instruction.
template <bool FP4>
struct StepShape {
    static constexpr int BN = FP4 ? kBN4 : kBN;
    static constexpr int StageB = BN * kBK;
    static constexpr int Stages = 4;
    static constexpr uint32_t ColScale = 2 * BN;  // FP4 block scales (16 columns)
    static constexpr uint32_t Idesc =
        FP4 ? ptx::idesc_mxf4_e2m1(kBM, BN) : ptx::idesc_e4m3_f32(kBM, BN);
};

template <int BN, int kStages>
struct __align__(8) TcShared {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t accfull[2];
    uint64_t accempty[2];
    uint64_t drain;          // arrives once every MMA issued has completed
    int last_use[kStages];   // last use of each stage a copy was issued for
    uint32_t tmem_base;
    int abort;
    float red[4][BN];
    float tred[4][BN];
};

template <bool FP4>
constexpr size_t step_smem_bytes()
{
    return 1024 /* alignment slack */ +
           (size_t)StepShape<FP4>::Stages * (kStageA + StepShape<FP4>::StageB) +
           sizeof(TcShared<StepShape<FP4>::BN, StepShape<FP4>::Stages>);
}
static_assert(step_smem_bytes<false>() <= 232448, "shared memory per CTA is limited to 227 KB");
static_assert(step_smem_bytes<true>() <= 232448, "shared memory per CTA is limited to 227 KB");
static_assert(2 * kBN <= (int)kTmemCols && 2 * kBN4 + 32 <= (int)kTmemCols,
              "accumulators and block scales exceed tensor memory");

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

// Bounded wait by every lane; false in all lanes if any gave up.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, int *abort, int *err)
{
    const bool ok = ptx::mbar_wait(bar, parity, abort, err);
    return __all_sync(0xFFFFFFFFu, ok);
}

template <bool FP4>
__device__ __forceinline__ void mma_elect(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate, uint32_t tmem_scale)
{
    if (FP4)
        ptx::mma_mxf4_elect(tmem_d, adesc, bdesc, StepShape<true>::Idesc, tmem_scale, tmem_scale,
                            accumulate);
    else
        asm volatile(
            "{\n\t.reg .pred p, e;\n\t"
            "elect.sync _|e, 0xffffffff;\n\t"
            "setp.ne.b32 p, %3, 0;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %4, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(accumulate), "r"(StepShape<false>::Idesc)
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

}  // namespace


// Epilogue of one tile in the eight epilogue warps (lane = spin; each warp
// takes half of the tile's replica columns, 32 at a time): the accumulator,
// x and y from global memory, the pinned update (two replicas per packed
// binary32 operation), x' and y' in place, sgn(x') as the next operand (the
// signs of a replica column gathered by one ballot; lane l then stores the
// codes of column l as one row segment); on evaluation steps the
// per-replica partial sums of s_i f_i and, with a trace, of y_i(t_k)^2,
// through a transposed butterfly.
// kPair: the tile belongs to a CTA pair, whose even CTA completes this CTA's
// accumulator barrier and receives its release (cluster address accempty_c).
// valid = false (a pair's row block past Np): the accumulator is waited for
// and released, nothing is loaded or stored.  Returns false once the
// epilogue warps have decided to leave (a wait gave up).
template <bool FP4, int kBN, bool kPair, typename Sh>
__device__ __forceinline__ bool epilogue_tile(
    Sh *sh, int b, int j, uint32_t accempty_c, int mb, int r0, bool valid, uint32_t tmem, int q,
    int cbase, int et, int lane, bool reduce, uint64_t stream_once, int N, int Np, int Kp, int Rp,
    float *__restrict__ X, float *__restrict__ Y, uint8_t *__restrict__ Snext, float pk,
    const StepConsts &c, int energy, int energy_only, float *__restrict__ Epart,
    float *__restrict__ Tpart, int *__restrict__ err, const float *__restrict__ gvec)
{
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int m0 = mb * kBM;
    const int i0 = m0 + q * 32;                  // first spin of this warp
    const int i = valid ? i0 + lane : 0;         // spin of this thread
    const bool live = valid && i < N;
    // x and y of one 32-column chunk, fetched before any store of the
    // chunk (the first chunk before the accumulator wait): all loads
    // of a chunk are in flight together
    float xv[32], yv[32];
    auto fetch = [&](int col0) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
            const int r = r0 + col0 + jj;
            const size_t e = (size_t)(r < Rp ? r : 0) * Np + i;
            xv[jj] = valid ? ptx::ld_f32_hint(X + e, stream_once) : 0.f;
            yv[jj] = (energy_only || !valid) ? 0.f : ptx::ld_f32_hint(Y + e, stream_once);
        }
    };
    fetch(cbase);
    const bool ok = kPair ? ptx::mbar_wait_cluster(&sh->accfull[b], (uint32_t)(j >> 1) & 1u,
                                                   &sh->abort, err)
                          : ptx::mbar_wait(&sh->accfull[b], (uint32_t)(j >> 1) & 1u, &sh->abort,
                                           err);
    if (epi_bar_or(!ok))
        return false;
    ptx::tc_fence_after();
    const StepConsts2 k2 = step_consts2(c);
    const uint64_t pk2 = f2_pack(pk, pk);
    const uint32_t livem = __ballot_sync(0xFFFFFFFFu, live);  // bit l: spin i0 + l is live
    for (int cb = 0; cb < kBN / 2 / 32; ++cb) {
        const int col0 = cbase + cb * 32;
        const int rc = r0 + col0;  // replica of the chunk's first column
        uint32_t fr[32];
        ptx::tmem_ld32(tmem + lane_off + (uint32_t)(b * kBN + col0), fr);
        if (cb > 0)
            fetch(col0);
        ptx::tmem_ld_wait();
        uint32_t negm = 0u;  // lane l: bit s set when spin i0 + s of replica rc + l is negative
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            // partial sums over this warp's 32 spins of 16 columns:
            // s_i f_i (evaluations) and y_i(t_k)^2 (trace)
            float tv[16], t2v[16];
#pragma unroll
            for (int u = 0; u < 16; u += 2) {
                const int jj = hh * 16 + u;
                const int r = rc + jj;
                const bool in0 = valid && r < Rp;  // uniform over the warp
                const bool in1 = valid && r + 1 < Rp;
                const float f0 = __uint_as_float(fr[jj]), f1 = __uint_as_float(fr[jj + 1]);
                const float x0 = xv[jj], x1 = xv[jj + 1];
                float e0 = 0.f, e1 = 0.f, s0 = 0.f, s1 = 0.f;
                if (energy || energy_only) {
                    e0 = (live && in0) ? (x0 >= 0.f ? f0 : -f0) : 0.f;
                    e1 = (live && in1) ? (x1 >= 0.f ? f1 : -f1) : 0.f;
                }
                if (!energy_only) {
                    const float y0 = yv[jj], y1 = yv[jj + 1];
                    if (Tpart) {
                        s0 = in0 ? __fmul_rn(y0, y0) : 0.f;  // y_i(t_k)^2 (Eq. eq_TInst)
                        s1 = in1 ? __fmul_rn(y1, y1) : 0.f;
                    }
                    // two replicas per packed binary32 operation (the same
                    // bits as two scalar updates); the per-replica friction
                    // of the Nose-Hoover thermostat in place of gamma dt
                    StepConsts2 kr = k2;
                    if (gvec)
                        kr.g = f2_pack(in0 ? __ldg(gvec + r) : 0.f, in1 ? __ldg(gvec + r + 1) : 0.f);
                    float xn0, xn1;
                    uint64_t yn;
                    sb_update2(f2_pack(f0, f1), f2_pack(x0, x1), f2_pack(yv[jj], yv[jj + 1]), pk2,
                               kr, xn0, xn1, yn);
                    const size_t e = (size_t)r * Np + i;
                    if (in0) {
                        ptx::st_f32_hint(X + e, xn0, stream_once);
                        ptx::st_f32_hint(Y + e, __uint_as_float((uint32_t)yn), stream_once);
                    }
                    if (in1) {
                        ptx::st_f32_hint(X + e + Np, xn1, stream_once);
                        ptx::st_f32_hint(Y + e + Np, __uint_as_float((uint32_t)(yn >> 32)),
                                         stream_once);
                    }
                    const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, !(xn0 >= 0.f));
                    const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, !(xn1 >= 0.f));
                    negm = lane == jj ? b0 : negm;
                    negm = lane == jj + 1 ? b1 : negm;
                }
                tv[u] = e0;
                tv[u + 1] = e1;
                t2v[u] = s0;
                t2v[u + 1] = s1;
            }
            if (reduce) {
                // transposed butterfly: after the exchanges over lane
                // bits 4..1 (8 + 4 + 2 + 1 shuffles per quantity) and
                // one over bit 0, lane l holds the sum over all 32
                // lanes of column (l >> 1) & 15
#pragma unroll
                for (int m = 16, n = 8; m >= 2; m >>= 1, n >>= 1) {
                    const bool up = (lane & m) != 0;
#pragma unroll
                    for (int k = 0; k < n; ++k) {
                        const float sa = up ? tv[k] : tv[k + n];
                        const float sb = up ? t2v[k] : t2v[k + n];
                        const float ra = __shfl_xor_sync(0xFFFFFFFFu, sa, m);
                        const float rb = __shfl_xor_sync(0xFFFFFFFFu, sb, m);
                        tv[k] = (up ? tv[k + n] : tv[k]) + ra;
                        t2v[k] = (up ? t2v[k + n] : t2v[k]) + rb;
                    }
                }
                const float ta = tv[0] + __shfl_xor_sync(0xFFFFFFFFu, tv[0], 1);
                const float tb = t2v[0] + __shfl_xor_sync(0xFFFFFFFFu, t2v[0], 1);
                if ((lane & 1) == 0) {
                    const int col = col0 + hh * 16 + ((lane >> 1) & 15);
                    sh->red[q][col] = ta;
                    sh->tred[q][col] = tb;
                }
            }
        }
        // lane l writes the next operand's codes of replica rc + l for this
        // warp's 32 spins (padded spins 0): FP8 one byte per spin (32 bytes),
        // FP4 one nibble per spin, spin 2m in the low nibble of byte m (16 bytes)
        if (!energy_only && valid && rc + lane < Rp) {
            const uint32_t neg = negm & livem;
            if (FP4) {
                uint32_t w[4];
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    w[m] = (spread8_nibbles(livem >> (8 * m)) * kFp4PlusOne) |
                           (spread8_nibbles(neg >> (8 * m)) << 3);
                *reinterpret_cast<uint4 *>(Snext + (size_t)(rc + lane) * (Kp / 2) + (i0 >> 1)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            } else {
                uint32_t w[8];
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    w[m] = (spread4_bytes(livem >> (4 * m)) * kFp8PlusOne) |
                           (spread4_bytes(neg >> (4 * m)) << 7);
                uint4 *dst = reinterpret_cast<uint4 *>(Snext + (size_t)(rc + lane) * Np + i0);
                dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
    }
    // the accumulator is read: the MMA may start the tile after next
    ptx::tc_fence_before();
    __syncwarp();
    if (lane == 0) {
        if (kPair)
            ptx::mbar_arrive_cluster(accempty_c);
        else
            ptx::mbar_arrive(&sh->accempty[b]);
    }
    if (reduce) {
        epi_bar();
        if (valid && et < kBN && r0 + et < Rp) {
            if (energy || energy_only)
                Epart[(size_t)mb * Rp + r0 + et] =
                    sh->red[0][et] + sh->red[1][et] + sh->red[2][et] + sh->red[3][et];
            if (Tpart && !energy_only)
                Tpart[(size_t)mb * Rp + r0 + et] =
                    sh->tred[0][et] + sh->tred[1][et] + sh->tred[2][et] + sh->tred[3][et];
        }
        epi_bar();  // the next tile's partial sums overwrite red
    }
    return true;
}

// Snext: the next step's operand, FP8 bytes [Rp][Np] or packed FP4 [Rp][Kp/2]
// (Kp = Np rounded up to 256: Kp/2 bytes per row, the padding zero).
template <bool FP4>
__global__ void __launch_bounds__(kThreads, 1)
tc_step_kernel(const __grid_constant__ CUtensorMap tmapA,
               const __grid_constant__ CUtensorMap tmapB, int N, int Np, int Kp, int Rp, int nrb,
               int band, int ntiles, float *__restrict__ X, float *__restrict__ Y,
               uint8_t *__restrict__ Snext, float pk, StepConsts c, int energy, int energy_only,
               float *__restrict__ Epart, float *__restrict__ Tpart, int *__restrict__ err,
               const float *__restrict__ gvec)
{
    constexpr int kBN = StepShape<FP4>::BN;  // replicas per tile
    constexpr int kStageB = StepShape<FP4>::StageB;
    constexpr int kStages = StepShape<FP4>::Stages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = base;
    uint8_t *sB = base + (size_t)kStages * kStageA;
    TcShared<kBN, kStages> *sh =
        reinterpret_cast<TcShared<kBN, kStages> *>(sB + (size_t)kStages * kStageB);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nk = (FP4 ? Kp / 2 : Np) / kBK;  // 128-byte K chunks of a row
    // tiles of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(&sh->full[s], 1);
            ptx::mbar_init(&sh->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&sh->accfull[b], 1);
            ptx::mbar_init(&sh->accempty[b], kEpiWarps);
        }
        ptx::mbar_init(&sh->drain, 1);
        for (int s = 0; s < kStages; ++s)
            sh->last_use[s] = -1;
        sh->abort = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmapA);
        ptx::prefetch_tmap(&tmapB);
    }
    if (warp == kMmaWarp)
        ptx::tmem_alloc(&sh->tmem_base, kTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    if (FP4) {
        // unit block scales: UE8M0 0x7F (2^0) in 16 columns of every lane; the
        // scale reads of every instruction fall inside them
        if (warp >= kFirstEpi && warp < kFirstEpi + 4) {
            uint32_t one[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                one[j] = 0x7F7F7F7Fu;
            ptx::tmem_st16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + StepShape<FP4>::ColScale,
                           one);
            ptx::tmem_st_wait();
        }
        ptx::tc_fence_before();
        __syncthreads();
        ptx::tc_fence_after();
    }

    if (warp < kIssuers) {
        // ------------------------------------------------------- TMA issuers
        // Global chunk counter g runs over the K chunks of this CTA's tiles
        // and fills stage g % kStages.  Issuer warp w serves the stages s
        // with s % 2 == w % 2 (always the same ones, so its parity waits see
        // every phase of them in order) and loads J (w < 2) or S (w >= 2).
        // The J issuer posts the stage's expected bytes (its one arrival);
        // both boxes count against it.
        if (lane == 0) {
            const bool isA = warp < 2;
            const int total = my_tiles * nk;
            for (int g = 0; g < total; ++g) {
                const int s = g % kStages;
                if ((s & 1) != (warp & 1))
                    continue;
                const int j = g / nk;
                const int kc = g - j * nk;
                const int tile = blockIdx.x + j * gridDim.x;
                int mb, rb;
                tile_coords(tile, Np / kBM, nrb, band, mb, rb);
                // each tile starts its K loop at its own chunk, so the CTAs
                // that share J rows or S rows do not ask for the same lines
                // at the same time (the partial forces are exact integers:
                // the summation order does not matter)
                const int kq = kRotateK ? (kc + tile) % nk : kc;
                const uint32_t ph = (uint32_t)(g / kStages) & 1u;
                if (!ptx::mbar_wait(&sh->empty[s], ph ^ 1u, &sh->abort, err))
                    break;
                atomicMax(&sh->last_use[s], g / kStages);  // for the drain
                if (isA) {
                    ptx::mbar_expect_tx(&sh->full[s], (uint32_t)(kStageA + kStageB));
                    ptx::tma_load_2d(sA + (size_t)s * kStageA, &tmapA, kq * kBK, mb * kBM,
                                     &sh->full[s]);
                } else {
                    ptx::tma_load_2d(sB + (size_t)s * kStageB, &tmapB, kq * kBK, rb * kBN,
                                     &sh->full[s]);
                }
            }
        }
    } else if (warp == kMmaWarp) {
        // --------------------------------------------------------------- MMA
        const uint64_t adesc0 = ptx::sw128_desc(ptx::smem_u32(sA));
        const uint64_t bdesc0 = ptx::sw128_desc(ptx::smem_u32(sB));
        int g = 0;
        for (int j = 0; j < my_tiles; ++j) {
            const int b = j & 1;
            // the epilogue has read this accumulator's previous tile
            if (!warp_wait(&sh->accempty[b], (uint32_t)((j >> 1) & 1) ^ 1u, &sh->abort, err))
                break;
            ptx::tc_fence_after();
            const uint32_t dcol = tmem + (uint32_t)(b * kBN);
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc, ++g) {
                const int s = g % kStages;
                const uint32_t ph = (uint32_t)(g / kStages) & 1u;
                if (!warp_wait(&sh->full[s], ph, &sh->abort, err)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint64_t ad = adesc0 + (uint64_t)((s * kStageA) >> 4);
                const uint64_t bd = bdesc0 + (uint64_t)((s * kStageB) >> 4);
#pragma unroll
                for (int kk = 0; kk < kBK / 32; ++kk)
                    mma_elect<FP4>(dcol, ad + (uint64_t)((kk * 32) >> 4),
                                   bd + (uint64_t)((kk * 32) >> 4), (kc | kk) != 0 ? 1u : 0u,
                                   tmem + StepShape<FP4>::ColScale);
                commit_elect(&sh->empty[s]);
            }
            if (!ok)
                break;
            commit_elect(&sh->accfull[b]);
        }
        commit_elect(&sh->drain);  // arrives once every MMA issued has completed
    } else {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - kFirstEpi;           // 0..7
        const int q = warp & 3;                    // tensor-memory lane quadrant
        const int cbase = (ew >> 2) * (kBN / 2);   // this warp's 128 replica columns
        const int et = threadIdx.x - 32 * kFirstEpi;
        const bool reduce = energy || energy_only || Tpart;
        // x and y are read and written once per step: their lines go first
        // from L2, so that the S rows of the band, re-read by every row
        // block, stay
        const uint64_t stream_once = ptx::l2_evict_first_policy();
        for (int j = 0; j < my_tiles; ++j) {
            const int tile = blockIdx.x + j * gridDim.x;
            int mb, rb;
            tile_coords(tile, Np / kBM, nrb, band, mb, rb);
            if (!epilogue_tile<FP4, kBN, false>(sh, j & 1, j, 0u, mb, rb * kBN, true, tmem, q,
                                                cbase, et, lane, reduce, stream_once, N, Np, Kp,
                                                Rp, X, Y, Snext, pk, c, energy, energy_only,
                                                Epart, Tpart, err, gvec))
                break;
        }
    }

    // drain before tensor memory and shared memory are given up (every exit
    // path): the last copy into each stage has landed and every MMA has
    // completed, each wait bounded.  A stage whose last use was never armed
    // (the J issuer gave up first) waits out the bound, with the error word set.
    __syncthreads();
    if (threadIdx.x < kStages) {
        const int u = sh->last_use[threadIdx.x];
        if (u >= 0)
            ptx::mbar_drain(&sh->full[threadIdx.x], (uint32_t)u & 1u, err);
    }
    if (warp == kMmaWarp)
        ptx::mbar_drain(&sh->drain, 0u, err);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == kMmaWarp)
        ptx::tmem_dealloc(tmem, kTmemCols);
}

// ------------------------------------------------- CTA-pair one-step kernel ---
// The same step with the tile shared by a CTA pair (a cluster of two,
// tcgen05 cta_group::2): the pair's MMA is M = 256 spins (128 J rows in each
// CTA's shared memory) by N = BN replicas, whose S rows are split over the
// pair (BN / 2 in each CTA), and each CTA's tensor memory receives its own
// 128 spins x BN replicas.  A CTA then moves 16 KB of J and BN / 2 x 128 B
// of S per K chunk instead of 16 KB and BN x 128 B, for the same work, so the
// copy latency is covered at a lower ingress.  The even CTA arms each stage
// for both CTAs' copies and issues the MMAs; its commits arrive on both
// CTAs' barriers.  Roles (480 threads per CTA): warps 0-5 TMA issuers (warp w
// owns stage w: lane 0 copies J, lane 1 copies S), warp 6 the MMA (even CTA),
// warps 7-14 the epilogue of this CTA's 128 spins (as in tc_step_kernel).
// A pair of row blocks past Np (N rounded up to 128 blocks of an odd count)
// loads zeros beyond the last row of J and stores nothing for it.
namespace {

constexpr int kQStages = 6;
constexpr int kQIssuers = kQStages;  // one issuer warp per stage
constexpr int kQMmaWarp = kQIssuers;
constexpr int kQFirstEpi = kQMmaWarp + 1;
constexpr int kQThreads = 32 * kQFirstEpi + kEpiThreads;

template <bool FP4>
struct PairShape {
    static constexpr int BN = FP4 ? kBN4 : kBN;  // replicas per pair tile (MMA N)
    static constexpr int BH = BN / 2;             // S rows per CTA
    static constexpr int StageB = BH * kBK;
    static constexpr uint32_t ColScale = 2 * BN;  // FP4 block scales (16 columns)
    static constexpr uint32_t Idesc =
        FP4 ? ptx::idesc_mxf4_e2m1(2 * kBM, BN) : ptx::idesc_e4m3_f32(2 * kBM, BN);
};

template <int BN>
struct __align__(8) QShared {
    uint64_t full[kQStages];   // (even CTA) both CTAs' copies of the stage have landed
    uint64_t empty[kQStages];  // the pair's MMAs have read the stage
    uint64_t accfull[2];       // the accumulator holds the tile's force
    uint64_t accempty[2];      // (even CTA) both CTAs' epilogues have read it
    uint64_t drain;            // (even CTA) every MMA issued has completed
    uint32_t tmem_base;
    int abort;
    int copies[kQStages][2][2];  // (even CTA) uses copied: [stage][CTA][J, S]
    float red[4][BN];
    float tred[4][BN];
};

template <bool FP4>
constexpr size_t pair_smem_bytes()
{
    return 1024 + (size_t)kQStages * (kStageA + PairShape<FP4>::StageB) +
           sizeof(QShared<PairShape<FP4>::BN>);
}
static_assert(pair_smem_bytes<false>() <= 232448, "shared memory per CTA is limited to 227 KB");
static_assert(pair_smem_bytes<true>() <= 232448, "shared memory per CTA is limited to 227 KB");

__device__ __forceinline__ bool qwarp_wait(uint64_t *bar, uint32_t parity, int *abort, int *err)
{
    const bool ok = ptx::mbar_wait_cluster(bar, parity, abort, err);
    return __all_sync(0xFFFFFFFFu, ok);
}

}  // namespace

template <bool FP4>
__global__ void __launch_bounds__(kQThreads, 1)
tc_step_pair_kernel(const __grid_constant__ CUtensorMap tmapA,
                    const __grid_constant__ CUtensorMap tmapB, int N, int Np, int Kp, int Rp,
                    int nrb, int band, int ntiles, float *__restrict__ X, float *__restrict__ Y,
                    uint8_t *__restrict__ Snext, float pk, StepConsts c, int energy,
                    int energy_only, float *__restrict__ Epart, float *__restrict__ Tpart,
                    int *__restrict__ err, const float *__restrict__ gvec)
{
    constexpr int kBN = PairShape<FP4>::BN;
    constexpr int kBH = PairShape<FP4>::BH;
    constexpr int kStageB = PairShape<FP4>::StageB;
    constexpr uint32_t kStageBytes = 2u * (kStageA + kStageB);  // both CTAs' copies
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = base;
    uint8_t *sB = base + (size_t)kQStages * kStageA;
    QShared<kBN> *sh = reinterpret_cast<QShared<kBN> *>(sB + (size_t)kQStages * kStageB);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t h = ptx::cluster_ctarank();  // 0: the CTA that issues the pair's MMAs
    const int nblk = Np / kBM;
    const int nmb2 = (nblk + 1) >> 1;           // pair row blocks of 256 spins
    const int nk = (FP4 ? Kp / 2 : Np) / kBK;   // 128-byte K chunks of a row
    const int cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
    const int my_tiles = cl < ntiles ? (ntiles - 1 - cl) / ncl + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kQStages; ++s) {
            ptx::mbar_init(&sh->full[s], 1);  // armed by the even CTA for both
            ptx::mbar_init(&sh->empty[s], 1);
            sh->copies[s][0][0] = sh->copies[s][0][1] = 0;
            sh->copies[s][1][0] = sh->copies[s][1][1] = 0;
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&sh->accfull[b], 1);
            ptx::mbar_init(&sh->accempty[b], 2 * kEpiWarps);
        }
        ptx::mbar_init(&sh->drain, 1);
        sh->abort = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmapA);
        ptx::prefetch_tmap(&tmapB);
    }
    if (warp == kQMmaWarp)
        ptx::tmem_alloc_pair(&sh->tmem_base, kTmemCols);
    ptx::tc_fence_before();
    ptx::cluster_sync();  // both CTAs' barriers and tensor memory exist
    ptx::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    if (FP4) {
        // unit block scales in 16 columns of every lane of both CTAs, before
        // the first pair MMA reads them
        if (warp >= kQFirstEpi && warp < kQFirstEpi + 4) {
            uint32_t one[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                one[j] = 0x7F7F7F7Fu;
            ptx::tmem_st16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + PairShape<FP4>::ColScale,
                           one);
            ptx::tmem_st_wait();
        }
        ptx::tc_fence_before();
        ptx::cluster_sync();
        ptx::tc_fence_after();
    }

    if (warp < kQIssuers) {
        // ------------------------------------------------------- TMA issuers
        // Issuer w serves stage w (loads g = w, w + S, ...): lane 0 copies the
        // CTA's 128 J rows, lane 1 its half of the tile's S rows.  Every copy
        // counts on the even CTA's barrier of the stage, which the even CTA's
        // lane 0 arms for both CTAs' bytes; a copy that lands first takes the
        // transaction count below zero until then (it cannot belong to the
        // previous use: that use's MMAs had completed before the stage was free).
        if (lane < 2) {
            const bool jl = lane == 0;
            const int s = warp;
            const int total = my_tiles * nk;
            const uint32_t full_own = ptx::smem_u32(&sh->full[s]);
            const uint32_t full_c = h == 0 ? full_own : ptx::mapa_shared(full_own, 0u);
            int used = 0;
            for (int g = s; g < total; g += kQStages) {
                const int j = g / nk;
                const int kc = g - j * nk;
                const int tile = cl + j * ncl;
                int mb2, rb;
                tile_coords(tile, nmb2, nrb, band, mb2, rb);
                const int kq = kRotateK ? (kc + tile) % nk : kc;
                const int u = g / kQStages;
                if (!ptx::mbar_wait_cluster(&sh->empty[s], (uint32_t)(u & 1) ^ 1u, &sh->abort, err))
                    break;
                if (jl) {
                    if (h == 0)
                        ptx::mbar_expect_tx(&sh->full[s], kStageBytes);
                    ptx::tma_load_2d_pair(sA + (size_t)s * kStageA, &tmapA, kq * kBK,
                                          mb2 * 2 * kBM + (int)h * kBM, full_c);
                } else {
                    ptx::tma_load_2d_pair(sB + (size_t)s * kStageB, &tmapB, kq * kBK,
                                          rb * kBN + (int)h * kBH, full_c);
                }
                used = u + 1;
            }
            // the uses copied, for the drain (in the even CTA's shared memory)
            int *dst = &sh->copies[s][h][jl ? 0 : 1];
            if (h == 0)
                *(volatile int *)dst = used;
            else
                ptx::st_shared_cluster(ptx::mapa_shared(ptx::smem_u32(dst), 0u), used);
        }
    } else if (warp == kQMmaWarp) {
        // ------------------------------------------------ the pair's MMAs
        if (h == 0) {
            const uint64_t adesc0 = ptx::sw128_desc(ptx::smem_u32(sA));
            const uint64_t bdesc0 = ptx::sw128_desc(ptx::smem_u32(sB));
            int g = 0;
            for (int j = 0; j < my_tiles; ++j) {
                const int b = j & 1;
                // both CTAs' epilogues have read this accumulator's previous tile
                if (!qwarp_wait(&sh->accempty[b], (uint32_t)((j >> 1) & 1) ^ 1u, &sh->abort,
                                err))
                    break;
                ptx::tc_fence_after();
                const uint32_t dcol = tmem + (uint32_t)(b * kBN);
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++g) {
                    const int s = g % kQStages;
                    if (!qwarp_wait(&sh->full[s], (uint32_t)(g / kQStages) & 1u, &sh->abort,
                                    err)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint64_t ad = adesc0 + (uint64_t)((s * kStageA) >> 4);
                    const uint64_t bd = bdesc0 + (uint64_t)((s * kStageB) >> 4);
#pragma unroll
                    for (int kk = 0; kk < kBK / 32; ++kk) {
                        const uint32_t acc = (kc | kk) != 0 ? 1u : 0u;
                        if (FP4)
                            ptx::mma_mxf4_pair_elect(dcol, ad + (uint64_t)((kk * 32) >> 4),
                                                     bd + (uint64_t)((kk * 32) >> 4),
                                                     PairShape<FP4>::Idesc,
                                                     tmem + PairShape<FP4>::ColScale, acc);
                        else
                            ptx::mma_fp8_pair_elect(dcol, ad + (uint64_t)((kk * 32) >> 4),
                                                    bd + (uint64_t)((kk * 32) >> 4),
                                                    PairShape<FP4>::Idesc, acc);
                    }
                    const uint32_t e_own = ptx::smem_u32(&sh->empty[s]);
                    ptx::commit_pair_elect(e_own);
                    ptx::commit_pair_elect(ptx::mapa_shared(e_own, 1u));
                }
                if (!ok)
                    break;
                const uint32_t a_own = ptx::smem_u32(&sh->accfull[b]);
                ptx::commit_pair_elect(a_own);
                ptx::commit_pair_elect(ptx::mapa_shared(a_own, 1u));
            }
            // drain: every MMA issued by this warp has completed
            ptx::commit_pair_elect(ptx::smem_u32(&sh->drain));
            ptx::mbar_drain(&sh->drain, 0u, err);
            __syncwarp();
        }
    } else if (warp >= kQFirstEpi) {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - kQFirstEpi;          // 0..7
        const int q = warp & 3;                    // tensor-memory lane quadrant
        const int cbase = (ew >> 2) * (kBN / 2);   // this warp's replica columns
        const int et = threadIdx.x - 32 * kQFirstEpi;
        const bool reduce = energy || energy_only || Tpart;
        const uint64_t stream_once = ptx::l2_evict_first_policy();
        for (int j = 0; j < my_tiles; ++j) {
            const int tile = cl + j * ncl;
            int mb2, rb;
            tile_coords(tile, nmb2, nrb, band, mb2, rb);
            const int mb = 2 * mb2 + (int)h;  // this CTA's 128-spin row block
            const uint32_t accempty_c =
                ptx::mapa_shared(ptx::smem_u32(&sh->accempty[j & 1]), 0u);
            if (!epilogue_tile<FP4, kBN, true>(sh, j & 1, j, accempty_c, mb, rb * kBN, mb < nblk,
                                               tmem, q, cbase, et, lane, reduce, stream_once, N,
                                               Np, Kp, Rp, X, Y, Snext, pk, c, energy,
                                               energy_only, Epart, Tpart, err, gvec))
                break;
        }
    }

    // Every role of both CTAs has left its loop: no issuer copies any more.
    // The even CTA then waits for the last copies of each stage from either
    // CTA; a last use some of whose copies were never made is completed here
    // (copies of use u are made only after the pair's MMAs have read use
    // u - 1, so only the last use of a stage can be incomplete).  A second
    // cluster barrier keeps both CTAs' shared memory alive until then.
    ptx::tc_fence_before();
    ptx::cluster_sync();
    if (h == 0 && threadIdx.x < kQStages) {
        const int st = threadIdx.x;
        const int aL = sh->copies[st][0][0], bL = sh->copies[st][0][1];
        const int aP = sh->copies[st][1][0], bP = sh->copies[st][1][1];
        int U = aL > bL ? aL : bL;
        U = aP > U ? aP : U;
        U = bP > U ? bP : U;
        if (U > 0) {
            const uint32_t landing = (aL >= U ? kStageA : 0) + (bL >= U ? kStageB : 0) +
                                     (aP >= U ? kStageA : 0) + (bP >= U ? kStageB : 0);
            if (aL >= U) {
                // armed for both CTAs' copies: stand in for the missing ones
                if (landing < kStageBytes)
                    ptx::mbar_complete_tx(&sh->full[st], kStageBytes - landing);
            } else {
                // never armed: arm it for the copies that were made
                ptx::mbar_expect_tx(&sh->full[st], landing);
            }
            ptx::mbar_drain(&sh->full[st], (uint32_t)(U - 1) & 1u, err);
        }
    }
    ptx::cluster_sync();
    ptx::tc_fence_after();
    if (warp == kQMmaWarp)
        ptx::tmem_dealloc_pair(tmem, kTmemCols);
}

// ------------------------------------------------------------- host side ---

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn()
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

// 2-D uint8 map over a row-major [rows][cols] array, box = 128 bytes x box_rows,
// with the 128-byte swizzle (the layout the matrix descriptors describe) or
// without swizzle (plain tile stores).
bool encode_u8(CUtensorMap *m, const void *ptr, uint64_t rows, uint64_t cols, uint32_t box_rows,
               bool swizzle = true)
{
    EncodeTiledFn fn = get_encode_fn();
    if (!fn)
        return false;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15u) != 0 || (cols % 16u) != 0)
        return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(ptr), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 3-D view of the same [rows][cols] byte array: (byte within a 128-byte K
// chunk, row, K chunk) with strides (1, cols, 128).  One box of
// 128 x box_rows x chunks lands in shared memory as `chunks` consecutive
// 128-byte-swizzled [box_rows][128] tiles, so a single copy fetches several K
// chunks.  Chunks past the end read as zero.
bool encode_u8_3d(CUtensorMap *m, const void *ptr, uint64_t rows, uint64_t cols,
                  uint32_t box_rows, uint32_t chunks)
{
    EncodeTiledFn fn = get_encode_fn();
    if (!fn)
        return false;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15u) != 0 || (cols % 128u) != 0)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)kBK, rows, cols / kBK};
    const cuuint64_t strides[2] = {cols, (cuuint64_t)kBK};
    const cuuint32_t box[3] = {(cuuint32_t)kBK, box_rows, chunks};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(ptr), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

cudaError_t tc_fp8_plan_create(TcPlan **out, const uint8_t *J8, const uint8_t *S8a,
                               const uint8_t *S8b, int Np, int Rp)
{
    *out = nullptr;
    if (Np % kBM != 0 || Rp % 128 != 0)
        return cudaErrorInvalidValue;
    TcPlan *p = new TcPlan();
    p->Np = Np;
    p->Rp = Rp;
    if (!encode_u8(&p->mapA, J8, (uint64_t)Np, (uint64_t)Np, kBM) ||
        !encode_u8(&p->mapB[0], S8a, (uint64_t)Rp, (uint64_t)Np, 128) ||
        !encode_u8(&p->mapB[1], S8b, (uint64_t)Rp, (uint64_t)Np, 128) ||
        !encode_u8_3d(&p->mapA3, J8, (uint64_t)Np, (uint64_t)Np, kBM, 2) ||
        !encode_u8_3d(&p->mapB3[0], S8a, (uint64_t)Rp, (uint64_t)Np, 128, 2) ||
        !encode_u8_3d(&p->mapB3[1], S8b, (uint64_t)Rp, (uint64_t)Np, 128, 2) ||
        !encode_u8(&p->mapBw[0], S8a, (uint64_t)Rp, (uint64_t)Np, kBN) ||
        !encode_u8(&p->mapBw[1], S8b, (uint64_t)Rp, (uint64_t)Np, kBN) ||
        !encode_u8(&p->mapJ64, J8, (uint64_t)Np, (uint64_t)Np, 64) ||
        !encode_u8(&p->mapBq[0], S8a, (uint64_t)Rp, (uint64_t)Np, kBN / 2) ||
        !encode_u8(&p->mapBq[1], S8b, (uint64_t)Rp, (uint64_t)Np, kBN / 2)) {
        delete p;
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(tc_step_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_bytes<false>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_step_pair_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_smem_bytes<false>());
    if (e != cudaSuccess) {
        delete p;
        return e;
    }
    *out = p;
    return cudaSuccess;
}

cudaError_t tc_fp4_plan_create(TcPlan **out, const uint8_t *J4, const uint8_t *S4a,
                               const uint8_t *S4b, int Np, int Kp, int Rp)
{
    *out = nullptr;
    if (Np % kBM != 0 || Kp % 256 != 0 || Kp < Np || Rp % 128 != 0)
        return cudaErrorInvalidValue;
    TcPlan *p = new TcPlan();
    p->Np = Np;
    p->Rp = Rp;
    p->Kp = Kp;
    // rows of Kp/2 bytes; a 128-byte box row holds 256 e2m1 values
    if (!encode_u8(&p->mapA, J4, (uint64_t)Np, (uint64_t)Kp / 2, kBM) ||
        !encode_u8_3d(&p->mapA3, J4, (uint64_t)Np, (uint64_t)Kp / 2, kBM, 2) ||
        !encode_u8_3d(&p->mapB3[0], S4a, (uint64_t)Rp, (uint64_t)Kp / 2, 128, 2) ||
        !encode_u8_3d(&p->mapB3[1], S4b, (uint64_t)Rp, (uint64_t)Kp / 2, 128, 2) ||
        !encode_u8(&p->mapBw[0], S4a, (uint64_t)Rp, (uint64_t)Kp / 2, kBN4) ||
        !encode_u8(&p->mapBw[1], S4b, (uint64_t)Rp, (uint64_t)Kp / 2, kBN4) ||
        !encode_u8(&p->mapBq[0], S4a, (uint64_t)Rp, (uint64_t)Kp / 2, kBN4 / 2) ||
        !encode_u8(&p->mapBq[1], S4b, (uint64_t)Rp, (uint64_t)Kp / 2, kBN4 / 2)) {
        delete p;
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(tc_step_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_bytes<true>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_step_pair_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_smem_bytes<true>());
    if (e != cudaSuccess) {
        delete p;
        return e;
    }
    *out = p;
    return cudaSuccess;
}

void tc_plan_destroy(TcPlan *p) { delete p; }

namespace {

template <bool FP4>
cudaError_t launch_step(cudaStream_t st, const TcPlan *plan, int parity, bool energy,
                        bool energy_only, int N, int Rp, float *X, float *Y, float pk,
                        StepConsts c, float *Epart, float *Tpart, uint8_t *Snext, int *err,
                        const float *gvec)
{
    // Rp (this run's padded replica count) may be below the capacity the
    // tensor maps were encoded for; Epart rows are Rp long.  A last tile that
    // reaches past Rp reads operand rows that are never stored back (past the
    // capacity the copy fills zeros).
    if (!plan || Rp % 128 != 0 || Rp > plan->Rp || (FP4 && plan->Kp < plan->Np))
        return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const size_t srow = FP4 ? (size_t)plan->Kp / 2 : (size_t)plan->Np;
    if (plan->Np >= kPairMinNp) {
        // CTA pairs over 256-spin x BN-replica tiles; clusters need not be
        // co-resident with one another
        constexpr int bn = PairShape<FP4>::BN;
        const int nrb = (Rp + bn - 1) / bn;
        const int nmb2 = (plan->Np / kBM + 1) / 2;
        const int ntiles = nmb2 * nrb;
        const int ncl = ntiles < sms / 2 ? ntiles : sms / 2;
        const size_t sbytes = (size_t)nrb * bn * srow;
        const int nbands = (int)((sbytes + kSBandBytes - 1) / kSBandBytes);
        const int band = (nrb + nbands - 1) / nbands;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * ncl, 1, 1);
        cfg.blockDim = dim3(kQThreads, 1, 1);
        cfg.dynamicSmemBytes = pair_smem_bytes<FP4>();
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, tc_step_pair_kernel<FP4>, plan->mapA,
                                  plan->mapBq[parity & 1], N, plan->Np, plan->Kp, Rp, nrb, band,
                                  ntiles, X, Y, Snext, pk, c, energy ? 1 : 0, energy_only ? 1 : 0,
                                  Epart, Tpart, err, gvec);
    }
    constexpr int bn = StepShape<FP4>::BN;
    const int nrb = (Rp + bn - 1) / bn;
    const int ntiles = (plan->Np / kBM) * nrb;
    const int grid = ntiles < sms ? ntiles : sms;
    // replica bands whose S rows fit the L2 budget, as few as possible
    const size_t sbytes = (size_t)nrb * bn * srow;
    const int nbands = (int)((sbytes + kSBandBytes - 1) / kSBandBytes);
    const int band = (nrb + nbands - 1) / nbands;
    tc_step_kernel<FP4><<<grid, kThreads, step_smem_bytes<FP4>(), st>>>(
        plan->mapA, plan->mapBw[parity & 1], N, plan->Np, plan->Kp, Rp, nrb, band, ntiles, X, Y,
        Snext, pk, c, energy ? 1 : 0, energy_only ? 1 : 0, Epart, Tpart, err, gvec);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_fp8_step(cudaStream_t st, const TcPlan *plan, int parity, bool energy,
                               bool energy_only, int N, int Rp, float *X, float *Y, float pk,
                               StepConsts c, float *Epart, float *Tpart, uint8_t *S8next,
                               int *err, const float *gvec)
{
    return launch_step<false>(st, plan, parity, energy, energy_only, N, Rp, X, Y, pk, c, Epart,
                              Tpart, S8next, err, gvec);
}

cudaError_t launch_tc_fp4_step(cudaStream_t st, const TcPlan *plan, int parity, bool energy,
                               bool energy_only, int N, int Rp, float *X, float *Y, float pk,
                               StepConsts c, float *Epart, float *Tpart, uint8_t *S4next,
                               int *err, const float *gvec)
{
    return launch_step<true>(st, plan, parity, energy, energy_only, N, Rp, X, Y, pk, c, Epart,
                             Tpart, S4next, err, gvec);
}

}  // namespace hsb
