// ALU rates of the device for the roofline of the ALU-bound kernels
// (qpfrg_alu_rates): ex2.approx, rcp.approx and FFMA results per SM per
// clock, each from one launch of eight independent dependency chains per
// thread on every SM (8 CTAs of 256 threads per SM), timed in SM clocks with
// clock64 (the longest CTA: all CTAs of an SM run concurrently).
#include "qpfrg_internal.h"

namespace {

constexpr int kChains = 8, kThreads = 256, kCtasPerSm = 8, kIters = 2048;

template <int OP>
__global__ void __launch_bounds__(kThreads) alu_rate_kernel(float *out, long long *cyc)
{
    float y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) y[c] = 0.1f * c + threadIdx.x * 1e-6f;
    const long long t0 = clock64();
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) {
                const float x = -y[c];     // 2^-y stays in (0, 1]
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y[c]) : "f"(x));
            } else if (OP == 1) {
                const float x = y[c] + 1.f;   // 1 / (1 + y) stays in (1/2, 1]
                asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y[c]) : "f"(x));
            } else {
                asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(y[c]) : "f"(0.999f), "f"(0.001f));
            }
        }
    }
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += y[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" qpfrg_status qpfrg_alu_rates(double *ex2_per_sm_clk, double *rcp_per_sm_clk, double *ffma_per_sm_clk)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
        cudaGetLastError();
        return QPFRG_ERR_CUDA;
    }
    const int blocks = sms * kCtasPerSm;
    float *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc((void **)&out, (size_t)blocks * kThreads * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&cyc, blocks * sizeof(long long)) != cudaSuccess) {
        cudaFree(out);
        cudaGetLastError();
        return QPFRG_ERR_OOM;
    }
    std::vector<long long> hc(blocks);
    double rate[3] = {0.0, 0.0, 0.0};
    qpfrg_status st = QPFRG_OK;
    for (int op = 0; op < 3 && st == QPFRG_OK; ++op) {
        // one launch to warm up, one measured
        for (int rep = 0; rep < 2; ++rep) {
            if (op == 0) alu_rate_kernel<0><<<blocks, kThreads>>>(out, cyc);
            else if (op == 1) alu_rate_kernel<1><<<blocks, kThreads>>>(out, cyc);
            else alu_rate_kernel<2><<<blocks, kThreads>>>(out, cyc);
        }
        if (cudaMemcpy(hc.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = QPFRG_ERR_CUDA;
            break;
        }
        long long cmax = 1;
        for (long long v : hc) cmax = v > cmax ? v : cmax;
        const double ops_per_sm = (double)kCtasPerSm * kThreads * kIters * kChains;
        rate[op] = ops_per_sm / (double)cmax;
    }
    cudaFree(out);
    cudaFree(cyc);
    if (cudaGetLastError() != cudaSuccess) st = QPFRG_ERR_CUDA;
    if (st != QPFRG_OK) return st;
    if (ex2_per_sm_clk) *ex2_per_sm_clk = rate[0];
    if (rcp_per_sm_clk) *rcp_per_sm_clk = rate[1];
    if (ffma_per_sm_clk) *ffma_per_sm_clk = rate[2];
    return QPFRG_OK;
}
