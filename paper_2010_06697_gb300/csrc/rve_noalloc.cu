// rve_stress_noalloc: the homogenised-stress reduction <W_F(F)> for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs inside a host application which owns every byte
// of device memory through its own pool and forbids further allocations (a fixed
// memory budget shared by many tenants), and latency-critical loops that must
// not call cudaMalloc/cudaFree because those calls may synchronise the device.
// Such callers hold F, the phase map and the material table in memory they
// already own and only need the reduction.
//
// The paper has no counterpart to this entry point; it is a systems addition.
//
// Scratch: the per-block partial sums and the last-block counter live in one
// file-scope static __device__ array (g_noalloc_scratch, 2 MiB + 256 B) that
// every GPU which loads this library keeps until the process exits.  Its device
// address is looked up once per device with cudaGetSymbolAddress, on the first
// call made with that device current; make that first call before any stream
// capture.  The address is kept for the life of the process, so this entry point
// must not be called on a device after cudaDeviceReset there.  All calls on a device share the array: the header (counter, error
// flag) is cleared at the start of every call, and calls whose work overlaps on
// the GPU race on it, so order them on one stream (or otherwise serialise them).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/rve.h"

namespace {

constexpr int kThreads = 128;
constexpr int kVoxelsPerBlock = 1024;                // 8 voxels per thread
constexpr int kMaxBlocks = 16384;                    // => at most 16,777,216 voxels (256^3)
constexpr int kSlots = 16;                           // >= d*d partial sums per block, 128-byte rows
constexpr int kHeader = 32;                          // doubles: counter, error flag, padding
constexpr long long kMaxVoxels = (long long)kMaxBlocks * kVoxelsPerBlock;
constexpr int kScratchDoubles = kHeader + kMaxBlocks * kSlots;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_ptr[256] = {};

// W_F for the two elastic laws of include/rve.h (written out here so that this
// file shares no code path with the solver's kernels).
template <int D, int MODEL>
__device__ __forceinline__ void piola(const double* F, double mu, double lam, double* P) {
    if (MODEL == RVE_NEOHOOKE) {
        double K[D * D], J;
        if (D == 2) {
            K[0] = F[3];
            K[1] = -F[2];
            K[2] = -F[1];
            K[3] = F[0];
            J = F[0] * F[3] - F[1] * F[2];
        } else {
            K[0] = F[4] * F[8] - F[5] * F[7];
            K[1] = F[5] * F[6] - F[3] * F[8];
            K[2] = F[3] * F[7] - F[4] * F[6];
            K[3] = F[2] * F[7] - F[1] * F[8];
            K[4] = F[0] * F[8] - F[2] * F[6];
            K[5] = F[1] * F[6] - F[0] * F[7];
            K[6] = F[1] * F[5] - F[2] * F[4];
            K[7] = F[2] * F[3] - F[0] * F[5];
            K[8] = F[0] * F[4] - F[1] * F[3];
            J = F[0] * K[0] + F[1] * K[1] + F[2] * K[2];
        }
        const double c = (lam * J * (J - 1.0) - mu) / J;  // P = mu F + (lam J (J-1) - mu) F^{-T}
        for (int p = 0; p < D * D; ++p) P[p] = mu * F[p] + c * K[p];
    } else {
        double tr = 0.0;
        for (int i = 0; i < D; ++i) tr += F[i * D + i] - 1.0;
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j)
                P[i * D + j] = mu * (F[i * D + j] + F[j * D + i] - (i == j ? 2.0 : 0.0)) + (i == j ? lam * tr : 0.0);
    }
}

template <int D, int MODEL>
__global__ void __launch_bounds__(kThreads)
k_stress_noalloc(const double* __restrict__ F, const uint8_t* __restrict__ phase, const double* __restrict__ params,
                 int nphase, int nparam, long long V, double* __restrict__ scratch, double* __restrict__ out) {
    constexpr int NN = D * D;
    __shared__ double s_sum[kThreads / 32][NN];
    __shared__ int s_last;
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
    unsigned int* bad = reinterpret_cast<unsigned int*>(scratch + 1);
    double acc[NN];
    for (int p = 0; p < NN; ++p) acc[p] = 0.0;
    const long long v0 = (long long)blockIdx.x * kVoxelsPerBlock;
    for (int t = threadIdx.x; t < kVoxelsPerBlock; t += kThreads) {
        const long long v = v0 + t;
        if (v >= V) break;
        const int ph = phase[v];
        if (ph >= nphase) {
            atomicOr(bad, 1u);
            continue;
        }
        double Fv[NN], P[NN];
        for (int p = 0; p < NN; ++p) Fv[p] = F[p * V + v];
        piola<D, MODEL>(Fv, params[ph * nparam + 0], params[ph * nparam + 1], P);
        for (int p = 0; p < NN; ++p) acc[p] += P[p];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = 0; p < NN; ++p) {
        double s = acc[p];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) s_sum[warp][p] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double* row = scratch + kHeader + (size_t)blockIdx.x * kSlots;
        for (int p = 0; p < NN; ++p) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += s_sum[w][p];
            row[p] = s;
        }
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int p = 0; p < NN; ++p) acc[p] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) {
        const double* row = scratch + kHeader + (size_t)b * kSlots;
        for (int p = 0; p < NN; ++p) acc[p] += __ldcg(row + p);
    }
    for (int p = 0; p < NN; ++p) {
        double s = acc[p];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) s_sum[warp][p] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const bool invalid = __ldcg(reinterpret_cast<const unsigned int*>(scratch + 1)) != 0u;
    for (int i = 0; i < 9; ++i) out[i] = 0.0;
    for (int p = 0; p < NN; ++p) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += s_sum[w][p];
        out[(p / D) * 3 + (p % D)] = invalid ? NAN : s / (double)V;
    }
    *counter = 0u;
}

// Device address of the scratch array for the current device (looked up once).
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return RVE_E_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RVE_E_CUDA;
        g_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_ptr[dev];
    return RVE_OK;
}

}  // namespace

extern "C" int rve_stress_noalloc(int dim, int n, int model, const double* F_dev, const uint8_t* phase_dev,
                                  const double* params_dev, int nphase, int nparam, double* S_dev, void* cuda_stream) {
    if ((dim != 2 && dim != 3) || n < 2 || n > 4096) return RVE_E_INVALID_ARG;
    if (model != RVE_NEOHOOKE && model != RVE_LINEAR) return RVE_E_INVALID_ARG;
    if (!F_dev || !phase_dev || !params_dev || !S_dev || nphase < 1 || nphase > 256 || nparam < 2)
        return RVE_E_INVALID_ARG;
    const long long V = dim == 3 ? (long long)n * n * n : (long long)n * n;
    if (V > kMaxVoxels) return RVE_E_INVALID_ARG;  // beyond the static scratch capacity
    double* scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc != RVE_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMemsetAsync(scratch, 0, kHeader * sizeof(double), st) != cudaSuccess) return RVE_E_CUDA;
    const int blocks = (int)((V + kVoxelsPerBlock - 1) / kVoxelsPerBlock);
    if (dim == 2 && model == RVE_NEOHOOKE)
        k_stress_noalloc<2, RVE_NEOHOOKE><<<blocks, kThreads, 0, st>>>(F_dev, phase_dev, params_dev, nphase, nparam,
                                                                       V, scratch, S_dev);
    else if (dim == 3 && model == RVE_NEOHOOKE)
        k_stress_noalloc<3, RVE_NEOHOOKE><<<blocks, kThreads, 0, st>>>(F_dev, phase_dev, params_dev, nphase, nparam,
                                                                       V, scratch, S_dev);
    else if (dim == 2)
        k_stress_noalloc<2, RVE_LINEAR><<<blocks, kThreads, 0, st>>>(F_dev, phase_dev, params_dev, nphase, nparam, V,
                                                                     scratch, S_dev);
    else
        k_stress_noalloc<3, RVE_LINEAR><<<blocks, kThreads, 0, st>>>(F_dev, phase_dev, params_dev, nphase, nparam, V,
                                                                     scratch, S_dev);
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_E_CUDA;
}
