// hsb_simt.cu -- CUDA-core kernels of libhsb: seeded initial state, the plain
// FP32 step (the comparison form), energy evaluation, best tracking, the
// Nose-Hoover xi update, the per-step trace reductions, the final energies of
// general couplings (exact fixed point, and binary64 for large N) and operand
// conversions.
//
// Paper: Kanao & Goto, arXiv 2203.08361.  Methods, Eqs. (eq_SyEuY),
// (eq_SyEuX), (eq_WallX), (eq_WallY), (eq_EuHeat); forces Eqs. (eq_fb),
// (eq_fd); energy Eq. (eq_Ising); instantaneous temperature Eq. (eq_TInst);
// Nose-Hoover Eqs. (eq_NH1), (eq_NH).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hsb_device.cuh"
#include "hsb_internal.cuh"

namespace hsb {

// ------------------------------------------------------------------ init ---

// x_i, y_i uniform in (-L, L) (Results, "SB with thermal fluctuation"), drawn
// from a counter-based SplitMix64 stream so that replica r's values depend on
// (seed, instance, r, i) only.
__global__ void init_kernel(uint64_t seed, uint32_t instance, float scale, int N, int Np, int R,
                            int Rp, float *__restrict__ X, float *__restrict__ Y,
                            uint8_t *__restrict__ S8, double *__restrict__ Ebest)
{
    const size_t total = (size_t)Rp * Np;
    const uint64_t s_inst = splitmix64_out(seed, (uint64_t)instance + 1u);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(e / Np);
        const uint32_t i = (uint32_t)(e % Np);
        float x = 0.f, y = 0.f;
        uint8_t s = 0;
        if ((int)i < N) {
            x = init_uniform(s_inst, r, i, 0, scale);
            y = init_uniform(s_inst, r, i, 1, scale);
            s = fp8_sign(x);
        }
        X[e] = x;
        Y[e] = y;
        if (S8)
            S8[e] = s;
        if (e < (size_t)R)
            Ebest[e] = INFINITY;
    }
}

cudaError_t launch_init(cudaStream_t st, uint64_t seed, uint32_t instance, float half_width,
                        int N, int Np, int R, int Rp, float *X, float *Y, uint8_t *S8,
                        double *Ebest)
{
    // scale = fl32(L * 2^-24), one rounding from binary64
    const float scale = (float)((double)half_width / 16777216.0);
    const size_t total = (size_t)Rp * Np;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    init_kernel<<<blocks, 256, 0, st>>>(seed, instance, scale, N, Np, R, Rp, X, Y, S8, Ebest);
    return cudaGetLastError();
}

// ------------------------------------------------------- plain FP32 step ---
//
// Tile: 128 spins (rows of J) x 128 replicas, 256 threads, 8 x 8 outputs per
// thread, K slices of 8 double-buffered in shared memory.  Every output keeps
// one accumulator updated by fmaf over k ascending, the binary32 reading of
// the force sum.  B operand element (r, k) is x_k of replica r (ballistic) or
// sgn(x_k) (discrete and energy evaluation), formed while staging the tile.

template <int FORM, bool ENERGY_ONLY>
__global__ void __launch_bounds__(256, 1)
simt_step_kernel(const float *__restrict__ J, int N, int Np, int Rp,
                 const float *__restrict__ Xcur, float *__restrict__ Xnext,
                 float *__restrict__ Y, float pk, StepConsts c, int energy,
                 float *__restrict__ Epart, float *__restrict__ Tpart,
                 const float *__restrict__ gvec)
{
    constexpr bool kSign = (FORM == 1) || ENERGY_ONLY;
    __shared__ __align__(16) float As[2][8][128];
    __shared__ __align__(16) float Bs[2][8][128];
    __shared__ float Ered[16][129];

    const int tid = threadIdx.x;
    const int tx = tid & 15;
    const int ty = tid >> 4;
    const int m0 = blockIdx.x * 128;
    const int r0 = blockIdx.y * 128;

    const int lrow = tid >> 1;
    const int lk = (tid & 1) * 4;
    const float *Ap = J + (size_t)(m0 + lrow) * Np + lk;
    const float *Bp = Xcur + (size_t)(r0 + lrow) * Np + lk;

    auto bval = [](float v) { return kSign ? (v >= 0.f ? 1.f : -1.f) : v; };

    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            acc[a][b] = 0.f;

    float4 ra = *reinterpret_cast<const float4 *>(Ap);
    float4 rb = *reinterpret_cast<const float4 *>(Bp);
    As[0][lk + 0][lrow] = ra.x;
    As[0][lk + 1][lrow] = ra.y;
    As[0][lk + 2][lrow] = ra.z;
    As[0][lk + 3][lrow] = ra.w;
    Bs[0][lk + 0][lrow] = bval(rb.x);
    Bs[0][lk + 1][lrow] = bval(rb.y);
    Bs[0][lk + 2][lrow] = bval(rb.z);
    Bs[0][lk + 3][lrow] = bval(rb.w);
    __syncthreads();

    const int nk = Np / 8;
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) {
            ra = *reinterpret_cast<const float4 *>(Ap + (size_t)(kt + 1) * 8);
            rb = *reinterpret_cast<const float4 *>(Bp + (size_t)(kt + 1) * 8);
        }
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[cur][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[cur][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        if (kt + 1 < nk) {
            const int nxt = cur ^ 1;
            As[nxt][lk + 0][lrow] = ra.x;
            As[nxt][lk + 1][lrow] = ra.y;
            As[nxt][lk + 2][lrow] = ra.z;
            As[nxt][lk + 3][lrow] = ra.w;
            Bs[nxt][lk + 0][lrow] = bval(rb.x);
            Bs[nxt][lk + 1][lrow] = bval(rb.y);
            Bs[nxt][lk + 2][lrow] = bval(rb.z);
            Bs[nxt][lk + 3][lrow] = bval(rb.w);
        }
        __syncthreads();
    }

    // Epilogue: thread owns rows {ty*4+a, 64+ty*4+a} and replicas
    // {tx*4+b, 64+tx*4+b}; one float4 of x and y per (replica, row group).
    float ep[8], tp[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int col = (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
        const size_t rowbase = (size_t)(r0 + col) * Np + m0;
        // per-replica friction factor of the Nose-Hoover thermostat
        StepConsts cr = c;
        if (gvec)
            cr.g = gvec[r0 + col];
        float e = 0.f, t2 = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ibase = h * 64 + ty * 4;
            const float4 x4 = *reinterpret_cast<const float4 *>(Xcur + rowbase + ibase);
            const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
            if (ENERGY_ONLY || energy) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float f = acc[h * 4 + a][b];
                    if (m0 + ibase + a < N)
                        e += (xv[a] >= 0.f ? f : -f);
                }
            }
            if (!ENERGY_ONLY) {
                const float4 y4 = *reinterpret_cast<const float4 *>(Y + rowbase + ibase);
                const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
                if (Tpart) {
#pragma unroll
                    for (int a = 0; a < 4; ++a)
                        t2 = __fadd_rn(t2, __fmul_rn(yv[a], yv[a]));
                }
                float xo[4], yo[4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    sb_update(acc[h * 4 + a][b], xv[a], yv[a], pk, cr, xo[a], yo[a]);
                *reinterpret_cast<float4 *>(Xnext + rowbase + ibase) =
                    make_float4(xo[0], xo[1], xo[2], xo[3]);
                *reinterpret_cast<float4 *>(Y + rowbase + ibase) =
                    make_float4(yo[0], yo[1], yo[2], yo[3]);
            }
        }
        ep[b] = e;
        tp[b] = t2;
    }
    if (!ENERGY_ONLY && Tpart) {
        // sum_i y_i(t_k)^2 of this row block per replica (Eq. eq_TInst)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int col = (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
            Ered[ty][col] = tp[b];
        }
        __syncthreads();
        if (tid < 128) {
            float sacc = 0.f;
            for (int t = 0; t < 16; ++t)
                sacc += Ered[t][tid];
            Tpart[(size_t)blockIdx.x * Rp + r0 + tid] = sacc;
        }
        __syncthreads();
    }
    if (ENERGY_ONLY || energy) {
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int col = (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
            Ered[ty][col] = ep[b];
        }
        __syncthreads();
        if (tid < 128) {
            float s = 0.f;
            for (int t = 0; t < 16; ++t)
                s += Ered[t][tid];
            Epart[(size_t)blockIdx.x * Rp + r0 + tid] = s;
        }
    }
}

cudaError_t launch_simt_step(cudaStream_t st, int form, bool energy_only, bool energy,
                             const float *J32, int N, int Np, int Rp, const float *Xcur,
                             float *Xnext, float *Y, float pk, StepConsts c, float *Epart,
                             float *Tpart, const float *gvec)
{
    dim3 grid(Np / 128, Rp / 128);
    if (energy_only)
        simt_step_kernel<1, true><<<grid, 256, 0, st>>>(J32, N, Np, Rp, Xcur, Xnext, Y, pk, c,
                                                         1, Epart, nullptr, nullptr);
    else if (form == 1)
        simt_step_kernel<1, false><<<grid, 256, 0, st>>>(J32, N, Np, Rp, Xcur, Xnext, Y, pk, c,
                                                          energy ? 1 : 0, Epart, Tpart, gvec);
    else
        simt_step_kernel<0, false><<<grid, 256, 0, st>>>(J32, N, Np, Rp, Xcur, Xnext, Y, pk, c,
                                                          0, Epart, Tpart, gvec);
    return cudaGetLastError();
}

// ------------------------------------------------- Nose-Hoover thermostat ---
// Eqs. (eq_NH1), (eq_NH): the friction -xi_r y_i takes the heating term's
// place in the update (factor g_r = -xi_r dt), and xi_r advances after the
// momenta from the updated ones.  Arithmetic in binary64 with the operations
// rounded one by one (no contraction), the factor rounded once to binary32.
// S_r = sum_i y_i^2 is formed in fixed point so that it does not depend on the
// order of summation: y_i is rounded to the nearest multiple of 2^-24 (exact
// for |y_i| >= 1/2), q_i = 2^24 y_i is squared as a 64-bit integer, the
// squares are added exactly in 128 bits, and 2^-48 times the total is rounded
// once to binary64.

// Padded replicas (R <= r < Rp) start from xi0 too: they carry real initial
// states, and on the persistent kernel they run the same thermostat, so they
// stay as stable as the reported replicas.
__global__ void nh_init_kernel(int R, int Rp, double xi0, double dt, double *__restrict__ xi,
                               float *__restrict__ gvec)
{
    (void)R;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Rp)
        return;
    xi[r] = xi0;
    gvec[r] = __double2float_rn(__dmul_rn(-xi0, dt));
}

namespace {

constexpr int kNhThreads = 128;  // one block per replica
constexpr int kNhBatch = 8;      // loads in flight per thread

__device__ __forceinline__ void add_u128(uint64_t &hi, uint64_t &lo, uint64_t bh, uint64_t bl)
{
    const uint64_t l = lo + bl;
    hi += bh + (l < lo ? 1ull : 0ull);
    lo = l;
}

// q^2 for q = round(2^24 y) (scaling exact, rounding to nearest even); |y|
// must stay below 256 (so |q| < 2^32), else *bad (also for NaN).
__device__ __forceinline__ void add_square_q24(float y, uint64_t &hi, uint64_t &lo, bool &bad)
{
    const float s = y * 16777216.0f;
    if (!(fabsf(s) < 4294967296.0f)) {
        bad = true;
        return;
    }
    const long long q = __float2ll_rn(s);
    const uint32_t a = (uint32_t)(q < 0 ? -q : q);
    add_u128(hi, lo, 0ull, (uint64_t)a * a);
}

// 2^-48 (hi 2^64 + lo) rounded once to binary64: the top 64 significant bits
// with the bits below them folded into a sticky bit 0 round to 53 bits as the
// full value does (the rounding position is bit 11 of the 64); the scaling
// by a power of two is exact.
__device__ __forceinline__ double u128_q48_to_double(uint64_t hi, uint64_t lo)
{
    if (hi == 0)
        return __dmul_rn(__ull2double_rn(lo), 0x1p-48);
    const int lz = __clzll((long long)hi);
    uint64_t t = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
    if (lo << lz)
        t |= 1ull;
    const double scale = __longlong_as_double((long long)(1023 + 16 - lz) << 52);  // 2^(16-lz)
    return __dmul_rn(__ull2double_rn(t), scale);
}

}  // namespace

// One block per replica; thread t takes i = t + 128 m, eight loads in flight
// at a time.  Integer sums are exact, so the split over threads, the xor tree
// and the combination of the warps do not change S.
__global__ void __launch_bounds__(kNhThreads)
nh_update_kernel(const float *__restrict__ Y, int N, int Np, double h, double NT, double dt,
                 double *__restrict__ xi, float *__restrict__ gvec, int *__restrict__ err)
{
    __shared__ uint64_t part[kNhThreads / 32][2];
    __shared__ int any_bad;
    const int r = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        any_bad = 0;
    const float *yr = Y + (size_t)r * Np;
    uint64_t hi = 0, lo = 0;
    bool bad = false;
    for (int i0 = threadIdx.x; i0 < N; i0 += kNhThreads * kNhBatch) {
        float v[kNhBatch];
#pragma unroll
        for (int u = 0; u < kNhBatch; ++u) {
            const int i = i0 + u * kNhThreads;
            v[u] = i < N ? yr[i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kNhBatch; ++u)
            add_square_q24(v[u], hi, lo, bad);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t oh = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
        const uint64_t ol = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        add_u128(hi, lo, oh, ol);
    }
    __syncthreads();  // any_bad is initialised
    if (bad)
        any_bad = 1;
    if (lane == 0) {
        part[w][0] = hi;
        part[w][1] = lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t sh = 0, sl = 0;
        for (int q = 0; q < kNhThreads / 32; ++q)
            add_u128(sh, sl, part[q][0], part[q][1]);
        if (any_bad)
            atomicExch(err, kErrRange);
        const double S = u128_q48_to_double(sh, sl);
        const double x = __dadd_rn(xi[r], __dmul_rn(h, __dsub_rn(S, NT)));
        xi[r] = x;
        gvec[r] = __double2float_rn(__dmul_rn(-x, dt));
    }
}

cudaError_t launch_nh_init(cudaStream_t st, int R, int Rp, double xi0, double dt, double *xi,
                           float *gvec)
{
    nh_init_kernel<<<(Rp + 255) / 256, 256, 0, st>>>(R, Rp, xi0, dt, xi, gvec);
    return cudaGetLastError();
}

cudaError_t launch_nh_update(cudaStream_t st, const float *Y, int N, int Np, int R, double h,
                             double NT, double dt, double *xi, float *gvec, int *err)
{
    nh_update_kernel<<<R, kNhThreads, 0, st>>>(Y, N, Np, h, NT, dt, xi, gvec, err);
    return cudaGetLastError();
}

// One trace entry (traced time t_k): over replicas r < R, E_r = -1/2 sum_b
// Epart[b][r] and T_r = (1/N) sum_b Tpart[b][r] (binary64, blocks in order);
// out = {min_r E_r, mean_r E_r, mean_r T_r}.  One block, fixed reduction order.
__global__ void __launch_bounds__(1024)
trace_reduce_kernel(const float *__restrict__ Epart, const float *__restrict__ Tpart, int nblk,
                    int N, int R, int Rp, double *__restrict__ out)
{
    __shared__ double smin[1024], ssum[1024], stt[1024];
    double mn = INFINITY, se = 0.0, st = 0.0;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        double e = 0.0, t = 0.0;
        for (int b = 0; b < nblk; ++b) {
            e += (double)Epart[(size_t)b * Rp + r];
            t += (double)Tpart[(size_t)b * Rp + r];
        }
        e = -0.5 * e;
        mn = fmin(mn, e);
        se += e;
        st += t / (double)N;
    }
    smin[threadIdx.x] = mn;
    ssum[threadIdx.x] = se;
    stt[threadIdx.x] = st;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + w]);
            ssum[threadIdx.x] += ssum[threadIdx.x + w];
            stt[threadIdx.x] += stt[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = smin[0];
        out[1] = ssum[0] / (double)R;
        out[2] = stt[0] / (double)R;
    }
}

// The same trace entry from many blocks.  Block b takes replicas 32 b ..
// 32 b + 31 (lane) and splits the row blocks over its 8 warps (warp w sums
// blocks w, w + 8, ... in order); warp 0 adds the 8 slices in order, reduces
// its 32 replicas with a fixed shuffle tree and writes part[3 b .. 3 b + 2] =
// {minimum E, sum E, sum T_inst}.  The last block to finish (ticket counter,
// reset by that block) combines the parts in a fixed order into out, so the
// result does not depend on the order in which blocks run.
__global__ void __launch_bounds__(256)
trace_parts_kernel(const float *__restrict__ Epart, const float *__restrict__ Tpart, int nblk,
                   int N, int R, int Rp, double *__restrict__ part, unsigned *__restrict__ ticket,
                   double *__restrict__ out)
{
    // entry blockIdx.y of a batch (one entry when gridDim.y == 1)
    {
        const size_t m = blockIdx.y;
        Epart += m * (size_t)nblk * Rp;
        Tpart += m * (size_t)nblk * Rp;
        part += m * 3 * (size_t)gridDim.x;
        ticket += m;
        out += 3 * m;
    }
    __shared__ double se_sh[8][32], st_sh[8][32];
    __shared__ double fmin_sh[256], fsum_sh[256], ftt_sh[256];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r = blockIdx.x * 32 + lane;
    double e = 0.0, t = 0.0;
    if (r < R) {
#pragma unroll 4
        for (int b = w; b < nblk; b += 8) {
            e += (double)Epart[(size_t)b * Rp + r];
            t += (double)Tpart[(size_t)b * Rp + r];
        }
    }
    se_sh[w][lane] = e;
    st_sh[w][lane] = t;
    __syncthreads();
    if (w == 0) {
        double es = 0.0, ts = 0.0;
        for (int v = 0; v < 8; ++v) {
            es += se_sh[v][lane];
            ts += st_sh[v][lane];
        }
        double mn = INFINITY, sm = 0.0, tt = 0.0;
        if (r < R) {
            mn = -0.5 * es;
            sm = -0.5 * es;
            tt = ts / (double)N;
        }
        for (int o = 16; o > 0; o >>= 1) {
            mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
            sm += __shfl_down_sync(0xffffffffu, sm, o);
            tt += __shfl_down_sync(0xffffffffu, tt, o);
        }
        if (lane == 0) {
            part[3 * (size_t)blockIdx.x] = mn;
            part[3 * (size_t)blockIdx.x + 1] = sm;
            part[3 * (size_t)blockIdx.x + 2] = tt;
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    double mn = INFINITY, sm = 0.0, tt = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += 256) {
        mn = fmin(mn, __ldcg(part + 3 * (size_t)q));
        sm += __ldcg(part + 3 * (size_t)q + 1);
        tt += __ldcg(part + 3 * (size_t)q + 2);
    }
    fmin_sh[threadIdx.x] = mn;
    fsum_sh[threadIdx.x] = sm;
    ftt_sh[threadIdx.x] = tt;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            fmin_sh[threadIdx.x] = fmin(fmin_sh[threadIdx.x], fmin_sh[threadIdx.x + h]);
            fsum_sh[threadIdx.x] += fsum_sh[threadIdx.x + h];
            ftt_sh[threadIdx.x] += ftt_sh[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = fmin_sh[0];
        out[1] = fsum_sh[0] / (double)R;
        out[2] = ftt_sh[0] / (double)R;
        *ticket = 0u;
    }
}

cudaError_t launch_trace_reduce_many(cudaStream_t st, const float *Epart, const float *Tpart,
                                     int nblk, int N, int R, int Rp, int entries, double *scratch,
                                     unsigned *tickets, double *out)
{
    // at most 65535 entries per launch (the grid's y extent)
    const int nparts = (R + 31) / 32;
    for (int m0 = 0; m0 < entries; m0 += 65535) {
        const int cnt = entries - m0 < 65535 ? entries - m0 : 65535;
        const size_t off = (size_t)m0 * nblk * Rp;
        trace_parts_kernel<<<dim3(nparts, cnt), 256, 0, st>>>(
            Epart + off, Tpart + off, nblk, N, R, Rp, scratch + (size_t)m0 * 3 * nparts,
            tickets + m0, out + (size_t)m0 * 3);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_trace_reduce(cudaStream_t st, const float *Epart, const float *Tpart, int nblk,
                                int N, int R, int Rp, double *scratch, unsigned *ticket,
                                double *out)
{
    if (!scratch || !ticket) {
        trace_reduce_kernel<<<1, 1024, 0, st>>>(Epart, Tpart, nblk, N, R, Rp, out);
        return cudaGetLastError();
    }
    trace_parts_kernel<<<(R + 31) / 32, 256, 0, st>>>(Epart, Tpart, nblk, N, R, Rp, scratch, ticket,
                                                      out);
    return cudaGetLastError();
}

// ------------------------------------------------------ best tracking ---

// E_r = -1/2 sum_b Epart[b][r] (binary64 sum over row blocks in order); a
// strictly lower energy replaces the best and copies sgn(x(t_k)).
__global__ void best_update_kernel(const float *__restrict__ Epart, int nblk, int N, int Np,
                                   int Rp, const float *__restrict__ X,
                                   const uint8_t *__restrict__ S8, double *__restrict__ Ebest,
                                   int8_t *__restrict__ Sbest, const uint8_t *__restrict__ S4,
                                   int Kp)
{
    const int r = blockIdx.x;
    __shared__ int take;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b)
            s += (double)Epart[(size_t)b * Rp + r];
        const double E = -0.5 * s;
        take = E < Ebest[r];
        if (take)
            Ebest[r] = E;
    }
    __syncthreads();
    if (!take)
        return;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        int8_t sp;
        if (X)
            sp = X[(size_t)r * Np + i] >= 0.f ? 1 : -1;
        else if (S4)
            sp = ((S4[(size_t)r * (Kp / 2) + (i >> 1)] >> (4 * (i & 1))) & 15u) == kFp4PlusOne ? 1
                                                                                           : -1;
        else
            sp = S8[(size_t)r * Np + i] == kFp8PlusOne ? 1 : -1;
        Sbest[(size_t)r * N + i] = sp;
    }
}

cudaError_t launch_best_update(cudaStream_t st, const float *Epart, int nblk, int N, int Np,
                               int R, int Rp, const float *X, const uint8_t *S8,
                               double *Ebest, int8_t *Sbest, const uint8_t *S4, int Kp)
{
    best_update_kernel<<<R, 256, 0, st>>>(Epart, nblk, N, Np, Rp, X, S8, Ebest, Sbest, S4, Kp);
    return cudaGetLastError();
}

// ---------------------------------------------------- binary64 energy ---

// Eq. (eq_Ising) for general couplings: E = -1/2 sum_i s_i sum_j J_ij s_j,
// every term exact in binary64 (+/-J_ij), one warp per row, fixed reduction
// order.  One block per replica.
__global__ void __launch_bounds__(256)
final_energy_f64_kernel(const float *__restrict__ J, int N, int Np,
                        const int8_t *__restrict__ Sbest, double *__restrict__ Eout)
{
    extern __shared__ int8_t s_sh[];
    __shared__ double red[8];
    const int r = blockIdx.x;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        s_sh[i] = Sbest[(size_t)r * N + i];
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int i = warp; i < N; i += 8) {
        const float *row = J + (size_t)i * Np;
        double a = 0.0;
        for (int j = lane; j < N; j += 32) {
            const double v = (double)row[j];
            a += s_sh[j] > 0 ? v : -v;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0)
            acc += s_sh[i] > 0 ? a : -a;
    }
    if (lane == 0)
        red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w)
            s += red[w];
        Eout[r] = -0.5 * s;
    }
}

cudaError_t launch_final_energy_f64(cudaStream_t st, const float *J32, int N, int Np, int R,
                                    const int8_t *Sbest, double *Eout)
{
    final_energy_f64_kernel<<<R, 256, (size_t)N, st>>>(J32, N, Np, Sbest, Eout);
    return cudaGetLastError();
}

// The same energies for many replicas at once, in exact fixed point on the
// upper triangle: E = -sum_{i<j} J_ij s_i s_j (J symmetric, zero diagonal),
// with q_ij = round(J_ij 2^scale_exp) (|q_ij| < 2^40; exact unless J_ij has
// bits below 2^-scale_exp).  Block (t, g) takes replicas 32t .. 32t+31 (one
// per lane) and rows i = 8g + w, 8g + w + 8G, ... (w = warp); a warp converts
// each element of its row once and broadcasts it with a shuffle, so every
// element costs one 64-bit integer add per replica (negated for s_i != s_j).
// Bounds (N <= 6300): a row sum < 2^53, a thread's rows < 2^59, a block
// < 2^62; final_energy_sum_kernel adds the G groups exactly and rounds once.
constexpr int kFeGroups = 16;

__global__ void __launch_bounds__(256)
final_energy_part_kernel(const float *__restrict__ J, int N, int Np, int R,
                         const int8_t *__restrict__ Sbest, double scale,
                         long long *__restrict__ part)
{
    extern __shared__ uint8_t neg_sh[];  // [N + 32][32]: 1 where s = -1 (0 past N)
    __shared__ long long red[8][32];
    const int r0 = blockIdx.x * 32;
    const int G = gridDim.y;
    for (int e = threadIdx.x; e < (N + 32) * 32; e += blockDim.x) {
        const int j = e >> 5, rr = e & 31;
        const int r = r0 + rr;
        neg_sh[e] = (j < N && r < R && Sbest[(size_t)r * N + j] < 0) ? 1 : 0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    long long acc = 0;
    for (int i = blockIdx.y * 8 + warp; i < N; i += G * 8) {
        const uint32_t ni = neg_sh[i * 32 + lane];
        const float *row = J + (size_t)i * Np;
        long long a = 0;
        for (int j0 = i + 1; j0 < N; j0 += 32) {
            const int j = j0 + lane;
            // the power-of-two scaling is exact in binary64; one rounding to an integer
            const long long ql = j < N ? __double2ll_rn(__dmul_rn((double)row[j], scale)) : 0ll;
#pragma unroll 8
            for (int jj = 0; jj < 32; ++jj) {
                const long long q = __shfl_sync(0xffffffffu, ql, jj);
                const uint32_t flip = ni ^ neg_sh[(j0 + jj) * 32 + lane];
                a += flip ? -q : q;  // q_ij s_i s_j
            }
        }
        acc += a;
    }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && r0 + lane < R) {
        long long s = 0;
        for (int w = 0; w < 8; ++w)
            s += red[w][lane];
        part[(size_t)blockIdx.y * R + r0 + lane] = s;
    }
}

// E_r = -2^-scale_exp sum_g part[g][r]: each part (< 2^62 in magnitude) is
// split at bit 31, the halves summed exactly in 64 bits, and the total
// hi 2^31 + lo (two exact binary64 values) rounded once by their addition.
__global__ void final_energy_sum_kernel(const long long *__restrict__ part, int G, int R,
                                        double inv_scale, double *__restrict__ Eout)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R)
        return;
    long long hi = 0, lo = 0;
    for (int g = 0; g < G; ++g) {
        const long long v = part[(size_t)g * R + r];
        hi += v >> 31;  // floor division: v = (v >> 31) 2^31 + (v & (2^31 - 1))
        lo += v & 0x7FFFFFFFll;
    }
    const double t = __dadd_rn(__dmul_rn((double)hi, 2147483648.0), (double)lo);
    Eout[r] = -__dmul_rn(t, inv_scale);
}

size_t final_energy_part_doubles(int R) { return (size_t)kFeGroups * R; }

cudaError_t launch_final_energy_f64_parts(cudaStream_t st, const float *J32, int N, int Np, int R,
                                          const int8_t *Sbest, int scale_exp, double *part,
                                          double *Eout)
{
    const dim3 grid((R + 31) / 32, kFeGroups);
    const size_t smem = (size_t)(N + 32) * 32;
    if (smem > 200 * 1024)  // N above about 6300: one block per replica instead
        return launch_final_energy_f64(st, J32, N, Np, R, Sbest, Eout);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(final_energy_part_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    long long *ipart = reinterpret_cast<long long *>(part);
    final_energy_part_kernel<<<grid, 256, smem, st>>>(J32, N, Np, R, Sbest,
                                                      ldexp(1.0, scale_exp), ipart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    final_energy_sum_kernel<<<(R + 255) / 256, 256, 0, st>>>(ipart, kFeGroups, R,
                                                             ldexp(1.0, -scale_exp), Eout);
    return cudaGetLastError();
}

// ------------------------------------------------------- conversions ---

__global__ void sign_to_fp8_kernel(const float *__restrict__ X, int N, int Np, size_t total,
                                   uint8_t *__restrict__ S8)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % Np);
        S8[e] = i < N ? fp8_sign(X[e]) : (uint8_t)0;
    }
}

cudaError_t launch_sign_to_fp8(cudaStream_t st, const float *X, int N, int Np, int Rp,
                               uint8_t *S8)
{
    const size_t total = (size_t)Rp * Np;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    sign_to_fp8_kernel<<<blocks, 256, 0, st>>>(X, N, Np, total, S8);
    return cudaGetLastError();
}

__global__ void j_to_fp8_kernel(const float *__restrict__ J, size_t total, uint8_t *__restrict__ J8)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const float v = J[e];
        J8[e] = v > 0.f ? kFp8PlusOne : (v < 0.f ? kFp8MinusOne : (uint8_t)0);
    }
}

cudaError_t launch_j_to_fp8(cudaStream_t st, const float *J32, int Np, uint8_t *J8)
{
    const size_t total = (size_t)Np * Np;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    j_to_fp8_kernel<<<blocks, 256, 0, st>>>(J32, total, J8);
    return cudaGetLastError();
}

// Packed e2m1 operands: two values per byte, the even index in the low nibble.
__device__ __forceinline__ uint32_t fp4_nibble_of_coupling(float v)
{
    return v > 0.f ? kFp4PlusOne : (v < 0.f ? kFp4MinusOne : 0u);
}

__global__ void j_to_fp4_kernel(const float *__restrict__ J, int Np, int Kp, size_t total,
                                uint8_t *__restrict__ J4)
{
    const int bpr = Kp / 2;  // bytes per row
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t row = e / bpr;
        const int j = 2 * (int)(e % bpr);
        const uint32_t lo = j < Np ? fp4_nibble_of_coupling(J[row * Np + j]) : 0u;
        const uint32_t hi = j + 1 < Np ? fp4_nibble_of_coupling(J[row * Np + j + 1]) : 0u;
        J4[e] = (uint8_t)(lo | (hi << 4));
    }
}

cudaError_t launch_j_to_fp4(cudaStream_t st, const float *J32, int Np, int Kp, uint8_t *J4)
{
    const size_t total = (size_t)Np * (Kp / 2);
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    j_to_fp4_kernel<<<blocks, 256, 0, st>>>(J32, Np, Kp, total, J4);
    return cudaGetLastError();
}

__global__ void sign_to_fp4_kernel(const float *__restrict__ X, int N, int Np, int Kp,
                                   size_t total, uint8_t *__restrict__ S4)
{
    const int bpr = Kp / 2;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / bpr;
        const int i = 2 * (int)(e % bpr);
        const uint32_t lo = i < N ? (X[r * Np + i] >= 0.f ? kFp4PlusOne : kFp4MinusOne) : 0u;
        const uint32_t hi =
            i + 1 < N ? (X[r * Np + i + 1] >= 0.f ? kFp4PlusOne : kFp4MinusOne) : 0u;
        S4[e] = (uint8_t)(lo | (hi << 4));
    }
}

cudaError_t launch_sign_to_fp4(cudaStream_t st, const float *X, int N, int Np, int Kp, int Rp,
                               uint8_t *S4)
{
    const size_t total = (size_t)Rp * (Kp / 2);
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    sign_to_fp4_kernel<<<blocks, 256, 0, st>>>(X, N, Np, Kp, total, S4);
    return cudaGetLastError();
}

}  // namespace hsb
