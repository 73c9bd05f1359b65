// hsb_tc.cu -- tensor-core (tcgen05) step kernels of libhsb for sm_103a.
//
// Discrete heated SB with couplings in {-1, 0, +1} (HdSB; Kanao & Goto,
// arXiv 2203.08361, Eq. (eq_fd) and Methods): the force F = J sgn(X) of all
// replicas is one GEMM with M = spins, N = replicas, K = spins.  J and sgn(X)
// are FP8 e4m3 (+1 = 0x38, -1 = 0xB8, 0 = 0x00), every product is -1, 0 or +1
// and every partial sum an integer of magnitude < 2^24, so FP32 accumulation
// in tensor memory is exact and the force equals the integer J sgn(x).
//
// One CTA computes a 128-spin x 128-replica tile of F:
//   warp 0     TMA producer: J and S tiles (128 x 128 bytes, 128-byte swizzle)
//              into a ring of shared-memory stages;
//   warp 1     allocates tensor memory and issues tcgen05.mma (kind::f8f6f4,
//              M = 128, N = 128, K = 32 per instruction) from one lane;
//   warps 2-5  epilogue: tcgen05.ld of the accumulator (one spin per lane),
//              the pinned spin update of the Methods equations, x and y in
//              place, sgn(x') as the next step's FP8 operand, and on
//              evaluation steps the per-replica partial sums of s_i f_i.
// Every mbarrier wait is bounded (a wall-clock budget); a wait that gives up
// sets the error word, makes the other roles leave their loops, and the CTA
// frees its tensor memory before it exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsb_device.cuh"
#include "hsb_internal.cuh"

namespace hsb {

namespace {

constexpr int kBM = 128;            // spins per tile (MMA M, tensor-memory lanes)
constexpr int kBN = 128;            // replicas per tile (MMA N, accumulator columns)
constexpr int kBK = 128;            // K bytes per stage (one 128-byte swizzle row)
constexpr int kStages = 6;
constexpr int kStageA = kBM * kBK;  // 16 KB
constexpr int kStageB = kBN * kBK;  // 16 KB
constexpr int kThreads = 192;
constexpr int kTmemCols = 128;
constexpr unsigned long long kWaitBudgetNs = 2000000000ull;  // 2 s

struct __align__(8) TcShared {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t accfull;
    uint32_t tmem_base;
    int abort;
    float red[4][kBN];
    float tred[4][kBN];
};

constexpr size_t kSmemBytes = 1024 /* alignment slack */ + (size_t)kStages * (kStageA + kStageB) +
                              sizeof(TcShared);
static_assert(kSmemBytes <= 232448, "shared memory per CTA is limited to 227 KB");

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false (and sets
// the abort flag and the error word) when the budget runs out or another role
// has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, TcShared *sh,
                                          int *err)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (*(volatile int *)&sh->abort)
            return false;
        if (globaltimer() - t0 > kWaitBudgetNs) {
            *(volatile int *)&sh->abort = 1;
            atomicExch(err, kErrTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05 "matrix descriptor"): K-major tile
// whose rows are 128 bytes with the 128-byte swizzle, 8-row groups 1024 bytes
// apart.  Fields: start address >> 4 (bits 0-13), leading byte offset >> 4
// (bits 16-29, unused for this layout, set to 1), stride byte offset >> 4
// (bits 32-45), fixed value 1 (bits 46-47), swizzle mode 2 = 128-byte (bits
// 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor of kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B = E4M3
// (bits 7-9, 10-12 = 0), both K-major, N >> 3 at bits 17-22, M >> 4 at bits
// 24-28.
constexpr uint32_t kIdescFp8 = (1u << 4) | ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_fp8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 columns of 32-bit accumulator: register j holds column
// (col + j) of the lane of this thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j)
        v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void epilogue_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

}  // namespace

__global__ void __launch_bounds__(kThreads, 1)
tc_fp8_step_kernel(const __grid_constant__ CUtensorMap tmapA,
                   const __grid_constant__ CUtensorMap tmapB, int N, int Np, int Rp,
                   float *__restrict__ X, float *__restrict__ Y, uint8_t *__restrict__ S8next,
                   float pk, StepConsts c, int energy, int energy_only,
                   float *__restrict__ Epart, float *__restrict__ Tpart, int *__restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = base;
    uint8_t *sB = base + (size_t)kStages * kStageA;
    TcShared *sh = reinterpret_cast<TcShared *>(sB + (size_t)kStages * kStageB);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM;
    const int r0 = blockIdx.y * kBN;
    const int nk = Np / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        mbar_init(&sh->accfull, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sh->tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            for (int kc = 0; kc < nk; ++kc) {
                const int s = kc % kStages;
                const uint32_t ph = (uint32_t)(kc / kStages) & 1u;
                if (!mbar_wait(&sh->empty[s], ph ^ 1u, sh, err))
                    break;
                mbar_expect_tx(&sh->full[s], (uint32_t)(kStageA + kStageB));
                tma_load_2d(sA + (size_t)s * kStageA, &tmapA, kc * kBK, m0, &sh->full[s]);
                tma_load_2d(sB + (size_t)s * kStageB, &tmapB, kc * kBK, r0, &sh->full[s]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc) {
                const int s = kc % kStages;
                const uint32_t ph = (uint32_t)(kc / kStages) & 1u;
                if (!mbar_wait(&sh->full[s], ph, sh, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + (size_t)s * kStageA);
                const uint32_t b0 = smem_u32(sB + (size_t)s * kStageB);
#pragma unroll
                for (int kk = 0; kk < kBK / 32; ++kk)
                    mma_fp8(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), kIdescFp8,
                            (kc | kk) != 0 ? 1u : 0u);
                mma_commit(&sh->empty[s]);
            }
            if (ok)
                mma_commit(&sh->accfull);
        }
    } else {
        // Epilogue warps 2..5; warp w reads tensor-memory lanes 32*(w % 4)..+31.
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const int i = m0 + row;
        const bool live = i < N;
        const bool ok = mbar_wait(&sh->accfull, 0u, sh, err);
        tc_fence_after();
        if (ok) {
            for (int cb = 0; cb < kBN / 32; ++cb) {
                float f[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 32), f);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = cb * 32 + j;
                    const size_t e = (size_t)(r0 + col) * Np + i;
                    const float x0 = X[e];
                    float term = 0.f;
                    if (energy || energy_only)
                        term = live ? (x0 >= 0.f ? f[j] : -f[j]) : 0.f;
                    if (!energy_only) {
                        float xn, yn;
                        const float y0 = Y[e];
                        if (Tpart) {
                            // y_i(t_k)^2 of this row block, summed over lanes (Eq. eq_TInst)
                            float t2 = __fmul_rn(y0, y0);
#pragma unroll
                            for (int off = 16; off > 0; off >>= 1)
                                t2 += __shfl_xor_sync(0xffffffffu, t2, off);
                            if (lane == 0)
                                sh->tred[q][col] = t2;
                        }
                        sb_update(f[j], x0, y0, pk, c, xn, yn);
                        X[e] = xn;
                        Y[e] = yn;
                        S8next[e] = live ? fp8_sign(xn) : (uint8_t)0;
                    }
                    if (energy || energy_only) {
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1)
                            term += __shfl_xor_sync(0xffffffffu, term, off);
                        if (lane == 0)
                            sh->red[q][col] = term;
                    }
                }
            }
        }
        if (energy || energy_only || Tpart) {
            epilogue_bar();
            const int t = threadIdx.x - 64;  // 0..127
            if (ok && t < kBN && (energy || energy_only)) {
                const float s = sh->red[0][t] + sh->red[1][t] + sh->red[2][t] + sh->red[3][t];
                Epart[(size_t)blockIdx.x * Rp + r0 + t] = s;
            }
            if (ok && t < kBN && Tpart && !energy_only) {
                const float s = sh->tred[0][t] + sh->tred[1][t] + sh->tred[2][t] + sh->tred[3][t];
                Tpart[(size_t)blockIdx.x * Rp + r0 + t] = s;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
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
    if (Np % kBM != 0 || Rp % kBN != 0)
        return cudaErrorInvalidValue;
    TcPlan *p = new TcPlan();
    p->Np = Np;
    p->Rp = Rp;
    if (!encode_u8(&p->mapA, J8, (uint64_t)Np, (uint64_t)Np, kBM) ||
        !encode_u8(&p->mapB[0], S8a, (uint64_t)Rp, (uint64_t)Np, kBN) ||
        !encode_u8(&p->mapB[1], S8b, (uint64_t)Rp, (uint64_t)Np, kBN) ||
        !encode_u8_3d(&p->mapA3, J8, (uint64_t)Np, (uint64_t)Np, kBM, 2) ||
        !encode_u8_3d(&p->mapB3[0], S8a, (uint64_t)Rp, (uint64_t)Np, kBN, 2) ||
        !encode_u8_3d(&p->mapB3[1], S8b, (uint64_t)Rp, (uint64_t)Np, kBN, 2) ||
        !encode_u8(&p->mapSt[0], S8a, (uint64_t)Rp, (uint64_t)Np, kBN, false) ||
        !encode_u8(&p->mapSt[1], S8b, (uint64_t)Rp, (uint64_t)Np, kBN, false)) {
        delete p;
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(tc_fp8_step_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) {
        delete p;
        return e;
    }
    *out = p;
    return cudaSuccess;
}

void tc_plan_destroy(TcPlan *p) { delete p; }

cudaError_t launch_tc_fp8_step(cudaStream_t st, const TcPlan *plan, int parity, bool energy,
                               bool energy_only, int N, int Rp, float *X, float *Y, float pk,
                               StepConsts c, float *Epart, float *Tpart, uint8_t *S8next,
                               int *err)
{
    // Rp (this run's padded replica count) may be below the capacity the
    // tensor maps were encoded for; Epart rows are Rp long.
    if (!plan || Rp % kBN != 0 || Rp > plan->Rp)
        return cudaErrorInvalidValue;
    dim3 grid(plan->Np / kBM, Rp / kBN);
    tc_fp8_step_kernel<<<grid, kThreads, kSmemBytes, st>>>(
        plan->mapA, plan->mapB[parity & 1], N, plan->Np, Rp, X, Y, S8next, pk, c,
        energy ? 1 : 0, energy_only ? 1 : 0, Epart, Tpart, err);
    return cudaGetLastError();
}

}  // namespace hsb
