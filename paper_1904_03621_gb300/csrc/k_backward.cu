// Backward of the low spectrum (step A7).
//
// Eq. (1) (Sec. 2) is linear in J and h, so for L = sum_k g_k E(s^(k)) over
// the returned states s^(k):
//     dL/dJ_ij = sum_k g_k s_i^(k) s_j^(k)   (i < j),
//     dL/dh_i  = sum_k g_k s_i^(k).
// One block per instance; every thread owns pairs (i, j) and sums over k in
// ascending order in FP64 (deterministic).  Entries on or below the
// diagonal of dJ are written as zero.
#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kBackThreads = 256;

__global__ void __launch_bounds__(kBackThreads) backward_kernel(const unsigned long long* states, const double* g,
                                                                const int* n_arr, int S, const long long* J_off,
                                                                const long long* h_off, void* dJ, void* dh,
                                                                int out_f64)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* C = reinterpret_cast<unsigned long long*>(smem);
    double* w = reinterpret_cast<double*>(C + S);
    const int b = blockIdx.x;
    const int n = n_arr[b];
    if (n < 1 || n > kMaxN) return;
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        C[k] = states[(size_t)b * S + k];
        w[k] = g[(size_t)b * S + k];
    }
    __syncthreads();
    const long long jo = J_off[b], ho = h_off[b];
    for (int idx = threadIdx.x; idx < n * n + n; idx += blockDim.x) {
        double acc = 0.0;
        if (idx < n * n) {
            const int i = idx / n, j = idx % n;
            if (i < j)
                for (int k = 0; k < S; k++) {
                    const bool same = (((C[k] >> i) ^ (C[k] >> j)) & 1ull) == 0ull;   // s_i s_j = +1
                    acc += same ? w[k] : -w[k];
                }
            if (out_f64) static_cast<double*>(dJ)[jo + idx] = acc;
            else static_cast<float*>(dJ)[jo + idx] = (float)acc;
        } else {
            const int i = idx - n * n;
            for (int k = 0; k < S; k++) acc += ((C[k] >> i) & 1ull) ? w[k] : -w[k];
            if (out_f64) static_cast<double*>(dh)[ho + i] = acc;
            else static_cast<float*>(dh)[ho + i] = (float)acc;
        }
    }
}

}  // namespace

cudaError_t launch_backward(const unsigned long long* states, const double* g, const int* n, int B, int S,
                            const long long* J_off, const long long* h_off, void* dJ, void* dh, int out_f64,
                            cudaStream_t s)
{
    size_t smem = (size_t)S * 16;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(backward_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    backward_kernel<<<B, kBackThreads, smem, s>>>(states, g, n, S, J_off, h_off, dJ, dh, out_f64);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
