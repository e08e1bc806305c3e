// Issue-rate probe: the per-SM throughput of the instruction classes the
// enumeration kernels are built from, measured on the GPU that runs them.
// It is the denominator of the walk kernels' roofline (their work is counted
// in ALU lane-instructions per configuration).
//
// Each kernel runs one 1024-thread block per SM (the register count keeps a
// second block off the SM).  A thread advances 8 independent recurrences of
// 4 registers; every step writes x_t = op(x_{t-1}, x_{t-2}, x_{t-4}), so each
// new value depends on three values no earlier step combined and no two steps
// fold into one instruction.  128 steps per loop iteration.
// Every block reads its SM cycle counter around the loop; the host times the
// launch with CUDA events.
#include <cstdint>
#include <vector>

#include "bf.h"
#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeChains = 8;
constexpr int kProbeRounds = 4;     // ring rounds per loop iteration: 128 steps per iteration

enum ProbeOp { kOpIadd3 = 0, kOpLop3 = 1, kOpVmnmx = 2, kOpFfma = 3 };

template <int OP>
__device__ __forceinline__ unsigned probe_op(unsigned a, unsigned b, unsigned c, int parity)
{
    unsigned d;
    if constexpr (OP == kOpIadd3) {
        d = a + b + c;
    } else if constexpr (OP == kOpLop3) {
        asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));   // majority
    } else {
        // 16x2 minimum / maximum, alternating so that no step absorbs the next
        if (parity) asm volatile("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(c));
        else asm volatile("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(c));
        (void)b;
    }
    return d;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads, 1) alu_probe_kernel(int iters, unsigned seed,
                                                                     unsigned long long* cycles, unsigned* sink)
{
    unsigned x[kProbeChains][4];
#pragma unroll
    for (int c = 0; c < kProbeChains; c++)
#pragma unroll
        for (int r = 0; r < 4; r++) x[c][r] = splitmix64(seed + threadIdx.x * 64u + c * 4u + r) >> 7;
    __syncthreads();
    const unsigned long long t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kProbeRounds * 4; k++) {
            const int r = k & 3;
#pragma unroll
            for (int c = 0; c < kProbeChains; c++) {
                // x_t from x_{t-1}, x_{t-2}, x_{t-4}: the ring slot r holds x_{t-4}
                x[c][r] = probe_op<OP>(x[c][(r + 3) & 3], x[c][(r + 2) & 3], x[c][r], r & 1);
            }
        }
    }
    const unsigned long long t1 = clock64();
    __syncthreads();
    unsigned acc = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; c++)
#pragma unroll
        for (int r = 0; r < 4; r++) acc ^= x[c][r];
    if (acc == 0x9E3779B9u) sink[blockIdx.x] = acc;     // practically never: keeps the chains alive
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// x_t = x_{t-1} * a + x_{t-4}: two register operands and one constant (three register operands
// per FFMA measured 66 lanes per clock, a register-read limit rather than the FP32 pipe's)
__global__ void __launch_bounds__(kProbeThreads, 1) ffma_probe_kernel(int iters, unsigned seed, float a,
                                                                      unsigned long long* cycles, unsigned* sink)
{
    float x[kProbeChains][4];
#pragma unroll
    for (int c = 0; c < kProbeChains; c++)
#pragma unroll
        for (int r = 0; r < 4; r++) x[c][r] = 1.0f + (float)((seed + threadIdx.x + c * 4 + r) & 255) * 1e-6f;
    __syncthreads();
    const unsigned long long t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kProbeRounds * 4; k++) {
            const int r = k & 3;
#pragma unroll
            for (int c = 0; c < kProbeChains; c++)
                x[c][r] = __fmaf_rn(x[c][(r + 3) & 3], a, x[c][r]);
        }
    }
    const unsigned long long t1 = clock64();
    __syncthreads();
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < kProbeChains; c++)
#pragma unroll
        for (int r = 0; r < 4; r++) acc += x[c][r];
    if (acc == 12345.678f) sink[blockIdx.x] = 1u;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace bf

namespace {

// instructions per thread of one launch: the recurrence steps only.  The loop counter's add
// and compare (2 integer instructions per 128 steps) are left out, so the integer rates are
// understated by at most 1.6 %.
double probe_instructions(int iters)
{
    return (double)iters * 4.0 * bf::kProbeRounds * bf::kProbeChains;
}

}  // namespace

extern "C" bf_status bf_measure_issue_rates(void* workspace, size_t workspace_bytes, bf_issue_rates* out,
                                            void* stream_ptr)
{
    using namespace bf;
    if (!out || !workspace) return report(BF_EINVAL, "null argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return report(BF_ECUDA, cudaGetErrorString(e));
    const size_t need = (size_t)sms * (sizeof(unsigned long long) + sizeof(unsigned));
    if (workspace_bytes < need || workspace_bytes < bf_issue_rates_workspace_size())
        return report(BF_EWORKSPACE, "probe workspace smaller than bf_issue_rates_workspace_size()");
    auto* cycles = static_cast<unsigned long long*>(workspace);
    auto* sink = reinterpret_cast<unsigned*>(cycles + sms);
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    cudaEvent_t ev0, ev1;
    if ((e = cudaEventCreate(&ev0)) != cudaSuccess) return report(BF_ECUDA, cudaGetErrorString(e));
    if ((e = cudaEventCreate(&ev1)) != cudaSuccess) {
        cudaEventDestroy(ev0);
        return report(BF_ECUDA, cudaGetErrorString(e));
    }
    const int iters_int = 2048, iters_fp = 4096;
    double lanes[4] = {0, 0, 0, 0}, mhz_sum = 0.0;
    std::vector<unsigned long long> host_cycles((size_t)sms);
    bf_status st = BF_OK;
    for (int op = 0; op < 4 && st == BF_OK; op++) {
        const int iters = op == kOpFfma ? iters_fp : iters_int;
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && st == BF_OK; rep++) {     // the first launch warms clocks and caches
            e = cudaEventRecord(ev0, stream);
            if (e == cudaSuccess) {
                switch (op) {
                case kOpIadd3: alu_probe_kernel<kOpIadd3><<<sms, kProbeThreads, 0, stream>>>(iters, 1u, cycles, sink); break;
                case kOpLop3: alu_probe_kernel<kOpLop3><<<sms, kProbeThreads, 0, stream>>>(iters, 2u, cycles, sink); break;
                case kOpVmnmx: alu_probe_kernel<kOpVmnmx><<<sms, kProbeThreads, 0, stream>>>(iters, 3u, cycles, sink); break;
                default: ffma_probe_kernel<<<sms, kProbeThreads, 0, stream>>>(iters, 4u, 0.999f, cycles, sink); break;
                }
                count_launches(1);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(ev1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(host_cycles.data(), cycles, (size_t)sms * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) st = report(BF_ECUDA, cudaGetErrorString(e));
        }
        if (st != BF_OK) break;
        double cyc_sum = 0.0, cyc_max = 0.0;
        for (int b = 0; b < sms; b++) {
            cyc_sum += (double)host_cycles[(size_t)b];
            if ((double)host_cycles[(size_t)b] > cyc_max) cyc_max = (double)host_cycles[(size_t)b];
        }
        const double per_block = probe_instructions(iters) * kProbeThreads;   // lane-instructions
        lanes[op] = per_block / (cyc_sum / sms);
        mhz_sum += cyc_max / (ms * 1e3);
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (st != BF_OK) return st;
    out->sms = sms;
    out->sm_clock_mhz = mhz_sum / 4.0;
    out->iadd3_lanes_per_clk = lanes[kOpIadd3];
    out->lop3_lanes_per_clk = lanes[kOpLop3];
    out->vmnmx_lanes_per_clk = lanes[kOpVmnmx];
    out->ffma_lanes_per_clk = lanes[kOpFfma];
    return BF_OK;
}

extern "C" size_t bf_issue_rates_workspace_size(void) { return (size_t)1024 * 12; }
