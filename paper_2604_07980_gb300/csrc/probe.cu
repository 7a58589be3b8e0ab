// probe.cu -- integer-pipe throughput probe used for roofline denominators.
//
// Every SM runs one CTA of 1024 threads; each thread advances 8 independent
// chains of the probed instruction (0: 32-bit popcount, 1: 3-input xor,
// 2: packed fp16 greater-than mask, 3: 32-bit add, 4: 32-bit multiply-add,
// 5: packed fp16 fused multiply-add with saturation), and the
// CTA's SM-clock cycle count gives operations per clock per SM.  Inline PTX with
// volatile asm keeps the compiler from folding the chains.
#include <algorithm>
#include <vector>

#include "ctm_internal.cuh"
#include "match_common.cuh"

namespace ctm {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned popc_op(unsigned x)
{
    unsigned r;
    asm volatile("popc.b32 %0, %1;" : "=r"(r) : "r"(x));
    return r;
}

__device__ __forceinline__ unsigned hgt2_mask_op(unsigned x, unsigned y)
{
    unsigned r;
    asm volatile("set.gt.u32.f16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(y));
    return r;
}

__device__ __forceinline__ unsigned iadd_op(unsigned x, unsigned y)
{
    unsigned r;
    asm volatile("add.u32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(y));
    return r;
}

__device__ __forceinline__ unsigned imad_op(unsigned x, unsigned y, unsigned z)
{
    unsigned r;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
    return r;
}

__device__ __forceinline__ unsigned hfma2_sat_op(unsigned x, unsigned y, unsigned z)
{
    unsigned r;
    asm volatile("fma.rn.sat.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
    return r;
}

__device__ __forceinline__ unsigned xor3_op(unsigned x, unsigned y, unsigned z)
{
    unsigned r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
    return r;
}

__global__ void __launch_bounds__(kProbeThreads) int_probe_kernel(int kind, int iters,
                                                                  unsigned *sink,
                                                                  long long *cycles)
{
    unsigned v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 2654435761u + c * 40503u + blockIdx.x;
    const unsigned y = 0x9e3779b9u ^ blockIdx.x, z = 0x7f4a7c15u + threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    if (kind == 0) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = popc_op(v[c]);
        }
    } else if (kind == 1) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = xor3_op(v[c], y, z);
        }
    } else if (kind == 2) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = hgt2_mask_op(v[c], y);
        }
    } else if (kind == 3) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = iadd_op(v[c], y);
        }
    } else if (kind == 4) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = imad_op(v[c], y, z);
        }
    } else {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = hfma2_sat_op(v[c], y, z);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    unsigned acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += v[c];
    if (acc == 0x12345678u) sink[blockIdx.x] = acc;  // keeps the chains alive
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// One CTA waits on an mbarrier phase that nothing completes: no thread arrives
// and no copy is in flight, so the bounded wait gives up and flags it.
__global__ void wait_probe_kernel(int *flag)
{
    __shared__ uint64_t mbar;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    mbar_wait_bounded(&mbar, 0u, flag);
}

}  // namespace

cudaError_t run_wait_probe(int *expired, float *waited_ms)
{
    int *flag = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
        wait_probe_kernel<<<1, 32>>>(flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(waited_ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(expired, flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (flag) cudaFree(flag);
    return e;
}

cudaError_t run_int_probe(int kind, int iters, double *ops_per_clk_per_sm)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    unsigned *sink = nullptr;
    long long *cyc = nullptr;
    e = cudaMalloc(&sink, sizeof(unsigned) * sms);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&cyc, sizeof(long long) * sms);
    if (e != cudaSuccess) { cudaFree(sink); return e; }
    int_probe_kernel<<<sms, kProbeThreads>>>(kind, iters / 8 + 1, sink, cyc);  // warm-up
    int_probe_kernel<<<sms, kProbeThreads>>>(kind, iters, sink, cyc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    std::vector<long long> h(sms);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
    cudaFree(sink);
    cudaFree(cyc);
    if (e != cudaSuccess) return e;
    std::sort(h.begin(), h.end());
    const double med = (double)h[sms / 2];
    *ops_per_clk_per_sm = med > 0 ? (double)kProbeThreads * iters * kChains / med : 0.0;
    return cudaSuccess;
}

}  // namespace ctm
