// ms_alu_peaks: measured issue rates of the execution units that bound the library's ALU-bound kernels (the
// walk: integer multiplies and logic for Philox, FP32, special functions; the renderer: special functions for
// the signed distance and the decoders' Softplus; the decoders: FP32 and special functions).  These are the
// denominators of the roofline fractions the benchmark reports, measured instead of derived from unit counts.
//
// Each unit is timed with its own kernel: every thread runs 8 independent dependency chains of one
// instruction, so the warps keep the unit busy rather than waiting on latency, in a full-occupancy grid of
// (SMs x 8) blocks of 256 threads, long enough (tens of milliseconds) that launch overhead does not count.
// The instructions are issued through inline PTX so that the compiler neither folds nor reorders the chains.
// Rates are operations per second over the whole GPU at whatever SM clock the GPU runs (the caller samples
// the clock).
#include "ms_device.cuh"

namespace ms {
namespace peaks {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <int kOp>
__device__ __forceinline__ void step(float (&f)[kChains], uint32_t (&u)[kChains])
{
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        if constexpr (kOp == MS_PEAK_FFMA) {
            asm volatile("fma.rn.f32 %0, %0, 0f3F7FFFFE, 0f3A83126F;" : "+f"(f[j]));
        } else if constexpr (kOp == MS_PEAK_EX2) {
            asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(f[j]));   // stays in (0, inf]; rate is value-free
        } else if constexpr (kOp == MS_PEAK_LG2) {
            asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(f[j]));
        } else if constexpr (kOp == MS_PEAK_SIN) {
            asm volatile("sin.approx.ftz.f32 %0, %0;" : "+f"(f[j]));
        } else if constexpr (kOp == MS_PEAK_RSQRT) {
            asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(f[j]));
        } else if constexpr (kOp == MS_PEAK_IMAD) {
            asm volatile("mad.lo.u32 %0, %0, 1664525, 1013904223;" : "+r"(u[j]));
        } else if constexpr (kOp == MS_PEAK_LOP3) {
            asm volatile("lop3.b32 %0, %0, 0x9E3779B9, 0xBB67AE85, 0x96;" : "+r"(u[j]));
        } else {
            asm volatile("mul.hi.u32 %0, %0, 0xD2511F53;" : "+r"(u[j]));
        }
    }
}

template <int kOp>
__global__ void __launch_bounds__(kThreads) peak_kernel(int iters, float* __restrict__ sink)
{
    float f[kChains];
    uint32_t u[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        f[j] = 0.5f + 0.01f * (float)(threadIdx.x & 31) + 0.001f * (float)j;
        u[j] = threadIdx.x * 2654435761u + (uint32_t)j;
    }
#pragma unroll 1
    for (int i = 0; i < iters; i += 8) {
#pragma unroll
        for (int k = 0; k < 8; ++k) step<kOp>(f, u);
    }
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += f[j] + (float)(u[j] & 1u);
    sink[(size_t)blockIdx.x * kThreads + threadIdx.x] = acc;
}

using KernelFn = void (*)(int, float*);
constexpr KernelFn kKernels[MS_PEAK_COUNT] = {
    peak_kernel<MS_PEAK_FFMA>, peak_kernel<MS_PEAK_EX2>,  peak_kernel<MS_PEAK_LG2>,  peak_kernel<MS_PEAK_SIN>,
    peak_kernel<MS_PEAK_RSQRT>, peak_kernel<MS_PEAK_IMAD>, peak_kernel<MS_PEAK_LOP3>, peak_kernel<MS_PEAK_IMULHI>,
};
// iterations per thread: about 20-50 ms per kernel on a B300 (FFMA and integer logic issue 8x faster than the
// special-function unit)
constexpr int kIters[MS_PEAK_COUNT] = {1 << 16, 1 << 13, 1 << 13, 1 << 13, 1 << 13, 1 << 15, 1 << 16, 1 << 15};

}  // namespace peaks
}  // namespace ms

extern "C" size_t ms_alu_peaks_scratch_bytes(void)
{
    return (size_t)ms::num_sms() * 8 * ms::peaks::kThreads * sizeof(float);
}

extern "C" ms_status ms_alu_peaks(double* ops_per_s, void* scratch, size_t scratch_bytes, void* stream)
{
    MS_NVTX("ms_alu_peaks");
    using namespace ms::peaks;
    MS_CHECK_ARG(ops_per_s != nullptr, "ms_alu_peaks: null output");
    const size_t need = ms_alu_peaks_scratch_bytes();
    MS_CHECK_ARG(scratch != nullptr && scratch_bytes >= need,
                 "ms_alu_peaks: a device scratch of at least %zu bytes is required", need);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)ms::num_sms() * 8u;
    float* sink = static_cast<float*>(scratch);
    cudaEvent_t e0, e1;
    MS_CUDA(cudaEventCreate(&e0));
    MS_CUDA(cudaEventCreate(&e1));
    ms_status st = MS_OK;
    for (int op = 0; op < MS_PEAK_COUNT && st == MS_OK; ++op) {
        kKernels[op]<<<blocks, kThreads, 0, s>>>(kIters[op] / 8, sink);    // warm-up (clocks, caches)
        cudaEventRecord(e0, s);
        kKernels[op]<<<blocks, kThreads, 0, s>>>(kIters[op], sink);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = ms::cuda_status(e, "ms_alu_peaks");
            break;
        }
        float ms_ = 0.0f;
        cudaEventElapsedTime(&ms_, e0, e1);
        const double ops = (double)blocks * kThreads * (double)kIters[op] * kChains;
        ops_per_s[op] = ops / ((double)ms_ * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}
