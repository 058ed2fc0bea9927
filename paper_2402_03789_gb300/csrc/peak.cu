// FP32 ALU peak of the device: register-resident, dependency-free FMA chains.
//
// The FP32 path and the tensor-product phases run on the FP32 FMA pipe, so
// their roofline needs that pipe's throughput.  Each thread keeps NCH
// independent accumulators in registers and updates each one per iteration
// (acc = acc * b + c with b, c kernel arguments, so nothing folds); the grid is
// a multiple of the SM count with enough warps to hide the FMA latency.  The
// packed form issues fma.rn.f32x2 (two FP32 FMAs per instruction).
#include "internal.h"

namespace sn {

constexpr int PEAK_NCH = 16;          // independent chains per thread
constexpr int PEAK_THREADS = 256;

__global__ void __launch_bounds__(PEAK_THREADS) ffma_peak_kernel(float* out, float b, float c, int iters) {
    float acc[PEAK_NCH];
#pragma unroll
    for (int j = 0; j < PEAK_NCH; ++j) acc[j] = (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < PEAK_NCH; ++j) acc[j] = fmaf(acc[j], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < PEAK_NCH; ++j) s += acc[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ unsigned long long f2_as_u64(float2 v) {
    return *reinterpret_cast<unsigned long long*>(&v);
}

__global__ void __launch_bounds__(PEAK_THREADS) ffma2_peak_kernel(float* out, float b, float c, int iters) {
    unsigned long long acc[PEAK_NCH / 2];
#pragma unroll
    for (int j = 0; j < PEAK_NCH / 2; ++j) acc[j] = f2_as_u64(make_float2((float)(threadIdx.x + 2 * j), (float)j));
    const unsigned long long bb = f2_as_u64(make_float2(b, b)), cc = f2_as_u64(make_float2(c, c));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < PEAK_NCH / 2; ++j)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[j]) : "l"(bb), "l"(cc));
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < PEAK_NCH / 2; ++j) {
        const float2 v = *reinterpret_cast<const float2*>(&acc[j]);
        s += v.x + v.y;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace sn

using namespace sn;

extern "C" sevennet_status sevennet_fp32_peak(int32_t device, int32_t packed, int32_t iters, double* flop,
                                              double* ms) {
    SN_CHECK(flop && ms, SEVENNET_EINVAL, "null output pointer");
    SN_CHECK(iters > 0, SEVENNET_EINVAL, "iters must be positive");
    SN_ENTER(device);
    const int blocks = 4 * num_sms(device);           // 32 warps per SM
    float* out = nullptr;
    SN_CUDA(cudaMalloc(&out, (size_t)blocks * PEAK_THREADS * sizeof(float)));
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st = nullptr;
    sevennet_status rc = SEVENNET_OK;
    auto launch = [&]() {
        if (packed) ffma2_peak_kernel<<<blocks, PEAK_THREADS, 0, st>>>(out, 0.999999f, 1e-6f, iters);
        else ffma_peak_kernel<<<blocks, PEAK_THREADS, 0, st>>>(out, 0.999999f, 1e-6f, iters);
        count_launches(1);
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        set_error("stream or event creation failed");
        rc = SEVENNET_ECUDA;
    } else {
        launch();                                      // warm-up (clocks ramp, code loads)
        cudaEventRecord(a, st);
        launch();
        cudaEventRecord(b, st);
        float t = 0.0f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess) {
            set_error("peak kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = SEVENNET_ECUDA;
        } else {
            *ms = t;
            *flop = 2.0 * PEAK_NCH * (double)iters * blocks * PEAK_THREADS;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    return rc;
}
