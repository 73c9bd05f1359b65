// hsb_noalloc.cu -- hsb_run_fp32_noalloc: the plain FP32 heated SB run for
// small instances, working entirely in a fixed scratch array that the library
// reserves at load time, so that the call itself allocates nothing.
//
// Some callers cannot allocate device memory on demand: code that runs under
// a fixed device-memory budget owned by another allocator (a framework's
// caching pool, a serving process that sizes memory once at start-up), or
// code that must not call cudaMalloc / cudaFree because those calls
// synchronize the device and stall the work of other streams.  For them this
// entry point keeps every intermediate buffer in one file-scope __device__
// array of kScratchBytes (about 2.6 MB), held by every GPU that loads the
// library until the process exits.  The caller passes the couplings and the
// output buffers in device memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "hsb.h"
#include "hsb_internal.cuh"

namespace hsb {
namespace {

constexpr int kNoAllocMaxNp = 512;  // N <= 512
constexpr int kNoAllocMaxRp = 256;  // R <= 256
constexpr int kMaxDevices = 64;

// Scratch layout (byte offsets), every block 256-byte aligned.
constexpr size_t kOffJ = 0;                                                   // Np*Np float
constexpr size_t kOffX0 = kOffJ + (size_t)kNoAllocMaxNp * kNoAllocMaxNp * 4;  // Rp*Np float
constexpr size_t kOffX1 = kOffX0 + (size_t)kNoAllocMaxRp * kNoAllocMaxNp * 4;
constexpr size_t kOffY = kOffX1 + (size_t)kNoAllocMaxRp * kNoAllocMaxNp * 4;
constexpr size_t kOffEpart = kOffY + (size_t)kNoAllocMaxRp * kNoAllocMaxNp * 4;  // nblk*Rp float
constexpr size_t kOffEbest = kOffEpart + (size_t)(kNoAllocMaxNp / kTileM) * kNoAllocMaxRp * 4;
constexpr size_t kOffEfinal = kOffEbest + (size_t)kNoAllocMaxRp * 8;
constexpr size_t kOffSbest = kOffEfinal + (size_t)kNoAllocMaxRp * 8;  // Rp*N int8
constexpr size_t kScratchBytes = kOffSbest + (size_t)kNoAllocMaxRp * kNoAllocMaxNp;

static_assert(kOffX0 % 256 == 0 && kOffX1 % 256 == 0 && kOffY % 256 == 0 &&
                  kOffEpart % 256 == 0 && kOffEbest % 256 == 0 && kOffEfinal % 256 == 0 &&
                  kOffSbest % 256 == 0,
              "scratch blocks must stay 256-byte aligned");

// The scratch itself.  In host code this name is only a host-side stand-in
// for the device array; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device performs this set-up) and kept for
// the life of the process: it belongs to the context current at that time, so
// it is stale after cudaDeviceReset (stated in hsb.h).
cudaError_t scratch_address(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_ptr[dev] = ptr;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return cudaSuccess;
}

// Caller's dense N x N couplings into the zero-padded Np x Np scratch copy.
__global__ void pad_couplings_kernel(const float *__restrict__ J, int N, int Np,
                                     float *__restrict__ Jp)
{
    const size_t total = (size_t)Np * Np;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / Np);
        const int c = (int)(e % Np);
        Jp[e] = (r < N && c < N) ? J[(size_t)r * N + c] : 0.f;
    }
}

}  // namespace

// Defined in hsb_api.cu: records the message returned by hsb_last_error().
hsb_status report_error(hsb_status s, const char *msg);

}  // namespace hsb

using namespace hsb;

extern "C" HSB_API hsb_status hsb_run_fp32_noalloc(const float *J, int N, const hsb_params *p,
                                                   int R, int steps, uint64_t seed,
                                                   int8_t *best_spins, double *best_energy,
                                                   void *cuda_stream)
{
    if (!J || !p || !best_spins || !best_energy)
        return report_error(HSB_E_INVAL, "hsb_run_fp32_noalloc: a pointer argument is NULL");
    const int Np = round_up(N < 1 ? 1 : N, kTileM);
    const int Rp = round_up(R < 1 ? 1 : R, kTileR);
    if (N < 2 || Np > kNoAllocMaxNp || R < 1 || Rp > kNoAllocMaxRp)
        return report_error(HSB_E_INVAL,
                    "hsb_run_fp32_noalloc: needs 2 <= N <= 512 and 1 <= R <= 256 (the size of "
                    "its fixed scratch array)");
    if (steps < 1 || (p->form != HSB_BALLISTIC && p->form != HSB_DISCRETE) || !(p->a0 > 0.0) ||
        !(p->dt > 0.0) || !(p->gamma >= 0.0) || !(p->init_half_width > 0.0) ||
        !(p->c0 > 0.0) || p->eval_every < 0)
        return report_error(HSB_E_INVAL,
                    "hsb_run_fp32_noalloc: needs steps >= 1, a valid form, a0 > 0, dt > 0, "
                    "gamma >= 0, init_half_width > 0, eval_every >= 0 and an explicit c0 > 0");
    if (p->thermostat != HSB_HEAT_CONSTANT)
        return report_error(HSB_E_UNSUPPORTED,
                    "hsb_run_fp32_noalloc: constant heating only (no Nose-Hoover thermostat)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return report_error(HSB_E_NODEVICE, "hsb_run_fp32_noalloc: no usable CUDA device");
    }
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(dev, &base);
    if (e != cudaSuccess)
        return report_error(HSB_E_CUDA, "hsb_run_fp32_noalloc: cudaGetSymbolAddress failed");

    float *Jp = reinterpret_cast<float *>(base + kOffJ);
    float *X[2] = {reinterpret_cast<float *>(base + kOffX0),
                   reinterpret_cast<float *>(base + kOffX1)};
    float *Y = reinterpret_cast<float *>(base + kOffY);
    float *Epart = reinterpret_cast<float *>(base + kOffEpart);
    double *Ebest = reinterpret_cast<double *>(base + kOffEbest);
    double *Efinal = reinterpret_cast<double *>(base + kOffEfinal);
    int8_t *Sbest = reinterpret_cast<int8_t *>(base + kOffSbest);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    StepConsts c;
    c.c0 = (float)p->c0;
    c.dt = (float)p->dt;
    c.q = (float)(p->a0 * p->dt);
    c.g = (float)(p->gamma * p->dt);
    c.nz = -0.0f;
    const int nblk = Np / kTileM;

    // The scratch keeps the previous call's contents: the padded couplings,
    // the state and Ebest (+inf) are rewritten in full before use.
    pad_couplings_kernel<<<64, 256, 0, st>>>(J, N, Np, Jp);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_init(st, seed, p->instance, (float)p->init_half_width, N, Np, R, Rp, X[0], Y,
                        nullptr, Ebest);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        // p_k = a0 - a(t_k), a(t_k) = a0 k / Ns, binary64 then rounded once
        double t = p->a0 * (double)k;
        t = t / (double)steps;
        const float pk = (float)(p->a0 - t);
        const int cur = k & 1;
        const bool ev = p->eval_every > 0 && k > 0 && k % p->eval_every == 0;
        if (ev && p->form == HSB_BALLISTIC)
            e = launch_simt_step(st, 1, true, true, Jp, N, Np, Rp, X[cur], nullptr, Y, 0.f, c,
                                 Epart, nullptr);
        if (e == cudaSuccess)
            e = launch_simt_step(st, p->form, false, ev && p->form == HSB_DISCRETE, Jp, N, Np, Rp,
                                 X[cur], X[cur ^ 1], Y, pk, c, Epart, nullptr);
        if (e == cudaSuccess && ev)
            e = launch_best_update(st, Epart, nblk, N, Np, R, Rp, X[cur], nullptr, Ebest, Sbest);
    }
    const int fin = steps & 1;
    if (e == cudaSuccess)
        e = launch_simt_step(st, 1, true, true, Jp, N, Np, Rp, X[fin], nullptr, Y, 0.f, c, Epart,
                             nullptr);
    if (e == cudaSuccess)
        e = launch_best_update(st, Epart, nblk, N, Np, R, Rp, X[fin], nullptr, Ebest, Sbest);
    if (e == cudaSuccess)
        e = launch_final_energy_f64(st, Jp, N, Np, R, Sbest, Efinal);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(best_spins, Sbest, (size_t)R * N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(best_energy, Efinal, (size_t)R * sizeof(double),
                            cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess)
        return report_error(HSB_E_CUDA, cudaGetErrorString(e));
    return HSB_OK;
}
