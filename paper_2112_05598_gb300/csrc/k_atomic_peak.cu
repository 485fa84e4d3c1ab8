// k_atomic_peak.cu -- microbenchmark of 16-byte global vector atomics on this
// GPU: the throughput that bounds the J^T scatter of A p, against which the
// benchmark reports that kernel.
#include <cuda_runtime.h>

#include "../../include/perf.h"
#include "perf_kernels.h"

namespace perf {
namespace {

constexpr long long kSlots = 1ll << 24;   // 16-byte slots: 256 MiB of scratch
constexpr int kBlocks = 152 * 8, kThreadsAP = 256, kIters = 200;

// Every lane adds a float4 to a slot shared by 32 / groups lanes of its warp;
// successive iterations move to another region so that L2 sees a spread of
// lines, as in a scatter over a large parameter vector.
__global__ void __launch_bounds__(kThreadsAP) k_vec_atomics(float* out, int groups) {
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int per = 32 / groups;
    for (int it = 0; it < kIters; ++it) {
        const long long base = (w * 1024 + (long long)it * 7919) % (kSlots - 64);
        const long long slot = base + (lane / per) * 2;   // < kSlots - 64 + 62
        atomicAdd(reinterpret_cast<float4*>(out) + slot, make_float4(1.f, 2.f, 3.f, 4.f));
    }
}

}  // namespace
}  // namespace perf

extern "C" perf_status perf_measure_atomic_peak(double* lane_ops_per_s) {
    if (!lane_ops_per_s) return PERF_ERR_INVALID_ARG;
    *lane_ops_per_s = 0.0;
    float* buf = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&buf, perf::kSlots * 16);
    if (e == cudaSuccess) e = cudaMemset(buf, 0, perf::kSlots * 16);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    double best = 0.0;
    const int groups[3] = {1, 4, 32};
    for (int g = 0; g < 3 && e == cudaSuccess; ++g) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // first run warms up
            cudaEventRecord(a);
            perf::k_vec_atomics<<<perf::kBlocks, perf::kThreadsAP>>>(buf, groups[g]);
            perf::count_launch();
            cudaEventRecord(b);
            e = cudaEventSynchronize(b);
            if (e == cudaSuccess) e = cudaGetLastError();
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            const double ops = (double)perf::kBlocks * perf::kThreadsAP * perf::kIters;
            if (e == cudaSuccess && rep == 1 && ms > 0.f && ops / (ms * 1e-3) > best)
                best = ops / (ms * 1e-3);
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) return PERF_ERR_CUDA;
    *lane_ops_per_s = best;
    return PERF_OK;
}
