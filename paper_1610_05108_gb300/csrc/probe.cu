// Throughput probes behind xyz_probe_peaks: the denominators of the
// rooflines reported for the integer kernels.  Each probe runs 8 independent
// dependency chains of one instruction per thread, 1024 threads on every SM,
// and is timed with CUDA events on the default stream; the SM clock during
// the launch is the mean clock64 cycle count of the blocks divided by the
// elapsed time.  The chains use inline PTX so that the compiler keeps one
// instruction per step: lop3.b32 (the integer ALU pipe, which also runs the
// shifts and byte permutations of the key transpose), add.u32 and popc.b32
// (the population count of the verification).
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/xyz.h"
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr int PR_THREADS = 1024;
constexpr int PR_CHAINS = 8;

template <int OP>
__global__ void __launch_bounds__(PR_THREADS, 1) peak_probe_kernel(uint32_t *sink, int iters, long long *cycles)
{
    uint32_t a[PR_CHAINS];
    const uint32_t b = threadIdx.x * 7u + 1u, c = blockIdx.x * 13u + 5u;
#pragma unroll
    for (int u = 0; u < PR_CHAINS; ++u)
        a[u] = threadIdx.x + (uint32_t)u * 0x9E3779B9u;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PR_CHAINS; ++u) {
            if (OP == 0)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[u]) : "r"(b), "r"(c));
            else if (OP == 1)
                asm volatile("add.u32 %0, %0, %1;" : "+r"(a[u]) : "r"(b));
            else
                asm volatile("popc.b32 %0, %0;" : "+r"(a[u]));
        }
    }
    const long long t1 = clock64();
    __syncthreads();
    uint32_t x = 0;
#pragma unroll
    for (int u = 0; u < PR_CHAINS; ++u)
        x ^= a[u];
    sink[blockIdx.x * PR_THREADS + threadIdx.x] = x;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace xyz

using namespace xyz;

extern "C" int xyz_probe_peaks(xyz_peaks *out)
{
    if (!out)
        return fail(XYZ_EINVAL, "null output");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0)
        return fail(XYZ_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
    uint32_t *sink = nullptr;
    long long *cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double rate[3] = {0, 0, 0}, mhz[3] = {0, 0, 0};
    const int iters[3] = {16384, 32768, 4096};   // about 1-2 ms per launch
    e = cudaMalloc(&sink, (size_t)sms * PR_THREADS * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMalloc(&cyc, (size_t)sms * sizeof(long long));
    if (e == cudaSuccess)
        e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    for (int op = 0; op < 3 && e == cudaSuccess; ++op) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the second launch is measured
            cudaEventRecord(e0, 0);
            if (op == 0)
                peak_probe_kernel<0><<<sms, PR_THREADS>>>(sink, iters[op], cyc);
            else if (op == 1)
                peak_probe_kernel<1><<<sms, PR_THREADS>>>(sink, iters[op], cyc);
            else
                peak_probe_kernel<2><<<sms, PR_THREADS>>>(sink, iters[op], cyc);
            cudaEventRecord(e1, 0);
            e = cudaEventSynchronize(e1);
            if (e == cudaSuccess)
                e = cudaGetLastError();
            if (e != cudaSuccess || rep == 0)
                continue;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            std::vector<long long> h((size_t)sms);
            e = cudaMemcpy(h.data(), cyc, (size_t)sms * sizeof(long long), cudaMemcpyDeviceToHost);
            double cy = 0.0;
            for (long long v : h)
                cy += (double)v;
            cy /= sms;
            const double ops = (double)sms * PR_THREADS * PR_CHAINS * iters[op];
            rate[op] = ops / (ms * 1e-3);
            mhz[op] = cy / (ms * 1e-3) / 1e6;
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(cyc);
    if (e != cudaSuccess)
        return fail(XYZ_ECUDA, std::string("peak probe: ") + cudaGetErrorString(e));
    out->alu_ops_per_s = rate[0];
    out->iadd_ops_per_s = rate[1];
    out->popc_ops_per_s = rate[2];
    out->sm_mhz = (mhz[0] + mhz[1] + mhz[2]) / 3.0;
    out->sms = sms;
    return XYZ_OK;
}
