/*
 * bte_noalloc.cu -- drift velocity and norm of caller-owned rows without any
 * device allocation.
 *
 * Some callers cannot allocate device memory when they need this reduction:
 * applications that hand all device memory to their own pool allocator and
 * account for every byte there, and latency-bound host paths that cannot
 * afford the device-wide synchronisation that cudaMalloc / cudaFree may
 * bring.  bte_observe_noalloc serves them: it is a variant of the
 * observables reduction of the step kernel (per-block partial sums, an
 * arrival ticket, the last block adding the partials in block order), whose
 * partials and ticket live in the file-scope array g_noalloc_scratch below
 * instead of in a handle's workspace.
 *
 * g_noalloc_scratch is a __device__ array: every GPU that loads this library
 * holds its kNoAllocScratchBytes until the process exits.  Host code must
 * not pass the array's name to a kernel (on the host it is only a stand-in);
 * its device address comes from cudaGetSymbolAddress, with the device
 * current, and is passed to the kernel.  The first call on a device does
 * that look-up; later calls outside stream capture repeat it (a cheap
 * runtime query, and the address changes when the caller resets the
 * device, which reloads the library's module), and calls during capture use
 * the address of the device's last call outside capture.
 */
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/bte.h"
#include "bte_device.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kColsPerBlock = 1024;
constexpr int kMaxBlocks = 1024;
/* largest m_points accepted: kMaxBlocks blocks of kColsPerBlock columns */
constexpr long long kMaxPoints = (long long)kMaxBlocks * kColsPerBlock;
/* partials [2][kMaxBlocks] doubles, then the arrival ticket */
constexpr size_t kTicketOffset = 2 * kMaxBlocks * sizeof(double);
constexpr size_t kNoAllocScratchBytes = kTicketOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

const double kPi = 3.14159265358979323846264338328;

template <typename T>
__global__ void observe_noalloc_kernel(const T* a0, const T* b1, int m_points, double vscale,
                                       double nscale, double* out, unsigned char* scratch) {
    __shared__ double red[32];
    double* part = reinterpret_cast<double*>(scratch);
    unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kTicketOffset);
    const int c0 = blockIdx.x * kColsPerBlock;
    const int c1 = min(c0 + kColsPerBlock, m_points);
    double sa = 0.0, sb = 0.0;
    for (int m = c0 + (int)threadIdx.x; m < c1; m += blockDim.x) {
        sa += (double)a0[m];
        sb += (double)b1[m];
    }
    const double ta = bte::dev::block_sum(sa, red);
    const double tb = bte::dev::block_sum(sb, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ta;
        part[kMaxBlocks + blockIdx.x] = tb;
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        if (t == gridDim.x - 1) {
            __threadfence();
            const volatile double* pv = part;
            double s_a = 0.0, s_b = 0.0;
            for (unsigned q = 0; q < gridDim.x; ++q) {
                s_a += pv[q];
                s_b += pv[kMaxBlocks + q];
            }
            out[0] = vscale * s_b;
            out[1] = nscale * s_a;
            *ticket = 0u;
        }
    }
}

/* Device address of g_noalloc_scratch on the current device: looked up
 * with the device current on every call outside stream capture (and cached
 * per device), taken from that cache while `s` is capturing. */
int scratch_address(cudaStream_t s, unsigned char** ptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BTE_ECUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return BTE_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cs == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return BTE_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *ptr = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return BTE_OK;
}

}  // namespace

extern "C" int bte_observe_noalloc(const bte_params* p, const void* a0_row, const void* b1_row,
                                   double* out, void* stream) {
    if (!p || !a0_row || !b1_row || !out) return BTE_EINVAL;
    if (p->m_points < 3 || p->m_points > kMaxPoints) return BTE_EINVAL;
    if (!(p->alpha > 0) || !std::isfinite(p->alpha) || !(p->phiy_max > p->phiy_min) ||
        !std::isfinite(p->phiy_min) || !std::isfinite(p->phiy_max))
        return BTE_EINVAL;
    if (p->precision != BTE_FP64 && p->precision != BTE_FP32_MIXED) return BTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* scratch = nullptr;
    int rc = scratch_address(s, &scratch);
    if (rc) return rc;
    /* the ticket must start at zero; a call that ended early may have left it set */
    if (cudaMemsetAsync(scratch + kTicketOffset, 0, sizeof(unsigned), s) != cudaSuccess)
        return BTE_ECUDA;
    const double dphi = (p->phiy_max - p->phiy_min) / (p->m_points - 1);
    const double sq = std::sqrt(p->alpha);
    const double vscale = kPi * sq * dphi, nscale = 2.0 * kPi * sq * dphi;
    const int blocks = (p->m_points + kColsPerBlock - 1) / kColsPerBlock;
    if (p->precision == BTE_FP64)
        observe_noalloc_kernel<double><<<blocks, kThreads, 0, s>>>(
            static_cast<const double*>(a0_row), static_cast<const double*>(b1_row), p->m_points,
            vscale, nscale, out, scratch);
    else
        observe_noalloc_kernel<float><<<blocks, kThreads, 0, s>>>(
            static_cast<const float*>(a0_row), static_cast<const float*>(b1_row), p->m_points,
            vscale, nscale, out, scratch);
    return cudaGetLastError() == cudaSuccess ? BTE_OK : BTE_ECUDA;
}
