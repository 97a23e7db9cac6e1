// Arithmetic peaks of the CUDA cores, measured: the denominators of the ALU
// rooflines of the FP32 stage kernels (the contraction is a chain of FP32
// fused multiply-adds; the double-float q0 of the z-forward pass is FP32
// arithmetic too) and of the FP64 form.  The paper has no counterpart: it
// reports no arithmetic rates.
//
// Each thread runs eight independent dependency chains of fused multiply-
// adds (enough independent work per warp to cover the pipe latency); the
// grid is eight 256-thread blocks per SM.  The result is fused multiply-adds
// per second times two (one multiply and one add each), from CUDA events
// around one launch after a warm-up launch.
#include <cuda_runtime.h>

#include "internal.h"

using namespace vdwgb;

namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

// KIND 0: scalar FP32 (fma.rn.f32); 1: two-lane FP32 (fma.rn.f32x2, two
// fused multiply-adds per instruction); 2: FP64 (fma.rn.f64)
template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int iters, float seed, int *sink) {
    if constexpr (KIND == 2) {
        double a[PROBE_CHAINS];
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (double)seed + 1e-3 * (threadIdx.x + k);
        const double m = 0.9999999, c = 1e-7;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], m, c);
        }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
        if (s == -1.0) atomicAdd(sink, 1);            // never true: keeps the chains live
    } else if constexpr (KIND == 1) {
        unsigned long long a[PROBE_CHAINS];
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k)
            a[k] = pack_f2(seed + 1e-3f * (float)(threadIdx.x + k), seed - 1e-3f * (float)k);
        const unsigned long long m = pack_f2(0.9999f, 0.9998f), c = pack_f2(1e-4f, 2e-4f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma_f2(a[k], m, c);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) {
            float lo, hi;
            unpack_f2(a[k], lo, hi);
            s += lo + hi;
        }
        if (s == -1.0f) atomicAdd(sink, 1);
    } else {
        float a[PROBE_CHAINS];
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = seed + 1e-3f * (float)(threadIdx.x + k);
        const float m = 0.9999f, c = 1e-4f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fmaf(a[k], m, c);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
        if (s == -1.0f) atomicAdd(sink, 1);
    }
}

template <int KIND>
cudaError_t launch_probe(int blocks, int iters, int *sink, cudaStream_t st) {
    k_fma_probe<KIND><<<blocks, PROBE_THREADS, 0, st>>>(iters, 0.5f, sink);
    return cudaGetLastError();
}

}  // namespace

extern "C" int vdwgb_alu_peak(int device, int kind, double *gflops) {
    if (!gflops || kind < 0 || kind > 2) return fail(VDWGB_EINVAL, "kind 0 (FP32), 1 (FP32x2) or 2 (FP64)");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(VDWGB_EINVAL, "no CUDA device %d", device);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_fail(e, "attribute");
    const int blocks = sms * PROBE_BLOCKS_PER_SM;
    // about 10 ms per launch at the expected rates (FP64: 1/64 of FP32)
    const int iters = kind == 2 ? 2000 : 60000;
    int *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    float ms = 0.f;
    e = cudaMalloc(&sink, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    auto run = [&]() {
        return kind == 0 ? launch_probe<0>(blocks, iters, sink, st)
                         : kind == 1 ? launch_probe<1>(blocks, iters, sink, st) : launch_probe<2>(blocks, iters, sink, st);
    };
    if (e == cudaSuccess) e = run();                       // warm-up (clocks up, code loaded)
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = run();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "ALU probe");
    const double fma_per_inst = kind == 1 ? 2.0 : 1.0;
    const double fmas = (double)blocks * PROBE_THREADS * PROBE_CHAINS * (double)iters * fma_per_inst;
    *gflops = 2.0 * fmas / (ms * 1e-3) / 1e9;
    return 0;
}
