// QUBO form of the problem (Sec. 2, Eqs. (2)-(3)) mapped exactly onto the
// Ising search.
//
// With q = (s + 1) / 2 and the library's sign (Eq. (2) negated, as Eq. (1)):
//     F(q) = sum_{i<j} a_ij q_i q_j + sum_i b_i q_i .
// Substituting q_i = (s_i + 1) / 2 and multiplying by 4 gives an Ising
// instance with J'_ij = a_ij and h'_i = 2 b_i + sum_{j != i} a_ij whose energy
// satisfies
//     4 F(q) = E'(s) + sum_{i<j} a_ij + 2 sum_i b_i ,
// i.e. the offset of Eq. (3) scaled by 4.  The scale keeps integer inputs
// integral, so the QUBO search is as exact as the Ising one; the ordering by
// (F, c) equals the ordering by (E', c).
//
// The two-state Potts model reduces the same way.  With s_i = 2 sigma_i - 1,
// [sigma_i == sigma_j] = (1 + s_i s_j) / 2 and h_i(sigma_i) = (h_i(0) + h_i(1)) / 2
// + s_i (h_i(1) - h_i(0)) / 2, so with J' = J and h'_i = h_i(1) - h_i(0)
//     2 E(sigma) = E'(s) + C,   C = sum_{i<j} J_ij + sum_i (h_i(0) + h_i(1)),
// and the configuration integer is the same (bit i set iff sigma_i = 1).
#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kQThreads = 256;

// strict-upper-triangle coupling a_ij (i != j) of a row-major matrix
template <typename T>
__device__ __forceinline__ T upper(const T* a, int n, int i, int j)
{
    return i < j ? a[i * n + j] : a[j * n + i];
}

// One block: J' (strict upper triangle copied, rest zero), h', and
// off4 = sum_{i<j} a_ij + 2 sum_i b_i summed in a fixed order.
template <typename T, typename TO, typename ACC>
__global__ void __launch_bounds__(kQThreads) qubo_prep_kernel(const T* a, const T* b, int n, TO* Jout, TO* hout,
                                                              ACC* off4, unsigned* flag)
{
    __shared__ ACC part[kQThreads];
    const int t = threadIdx.x;
    for (int idx = t; idx < n * n; idx += kQThreads) {
        const int i = idx / n, j = idx % n;
        Jout[idx] = i < j ? (TO)a[idx] : (TO)0;
    }
    ACC acc = 0;
    for (int i = t; i < n; i += kQThreads) {
        ACC hi = (ACC)2 * (ACC)b[i];
        for (int j = 0; j < n; j++)
            if (j != i) hi += (ACC)upper(a, n, i, j);
        ACC row = (ACC)2 * (ACC)b[i];
        for (int j = i + 1; j < n; j++) row += (ACC)a[i * n + j];
        acc += row;
        if (sizeof(TO) == 4 && sizeof(ACC) == 8 && (hi > (ACC)INT32_MAX || hi < (ACC)INT32_MIN))
            atomicOr(flag, 1u);           // integer field outside int32
        hout[i] = (TO)hi;
    }
    part[t] = acc;
    __syncthreads();
    for (int w = kQThreads / 2; w > 0; w >>= 1) {
        if (t < w) part[t] += part[t + w];
        __syncthreads();
    }
    if (t == 0) *off4 = part[0];
}

// Two-state Potts: J' (strict upper triangle), h'_i = h_i(1) - h_i(0) and C, one block.
template <typename T, typename TO, typename ACC>
__global__ void __launch_bounds__(kQThreads) potts2_prep_kernel(const T* J, const T* h, int n, TO* Jout, TO* hout,
                                                                ACC* cst, unsigned* flag)
{
    __shared__ ACC part[kQThreads];
    const int t = threadIdx.x;
    for (int idx = t; idx < n * n; idx += kQThreads) {
        const int i = idx / n, j = idx % n;
        Jout[idx] = i < j ? (TO)J[idx] : (TO)0;
    }
    ACC acc = 0;
    for (int i = t; i < n; i += kQThreads) {
        const ACC hi = (ACC)h[2 * i + 1] - (ACC)h[2 * i];
        ACC row = (ACC)h[2 * i] + (ACC)h[2 * i + 1];
        for (int j = i + 1; j < n; j++) row += (ACC)J[i * n + j];
        acc += row;
        if (sizeof(TO) == 4 && sizeof(ACC) == 8 && (hi > (ACC)INT32_MAX || hi < (ACC)INT32_MIN))
            atomicOr(flag, 1u);           // integer field outside int32
        hout[i] = (TO)hi;
    }
    part[t] = acc;
    __syncthreads();
    for (int w = kQThreads / 2; w > 0; w >>= 1) {
        if (t < w) part[t] += part[t + w];
        __syncthreads();
    }
    if (t == 0) *cst = part[0];
}

// E[k] = (E'[k] + C) / 2
__global__ void potts2_finish_i64_kernel(long long* E, int S, const long long* cst, unsigned* flag,
                                         const unsigned* map_flag)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0 && map_flag && *map_flag) atomicOr(flag, kErrRange);   // h' left int32: the search was void
    if (k >= S) return;
    const long long v = E[k] + *cst;
    if (v & 1ll) atomicOr(flag, 2u);       // cannot happen for a consistent instance
    E[k] = v / 2;
}

__global__ void potts2_finish_f64_kernel(double* E, int S, const double* cst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    E[k] = (E[k] + *cst) * 0.5;
}

// F[k] = (E'[k] + off4) / 4
__global__ void qubo_finish_i64_kernel(long long* F, int S, const long long* off4, unsigned* flag,
                                       const unsigned* map_flag)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0 && map_flag && *map_flag) atomicOr(flag, kErrRange);   // h' left int32: the search was void
    if (k >= S) return;
    const long long v = F[k] + *off4;
    if (v & 3ll) atomicOr(flag, 2u);       // cannot happen for a consistent instance
    F[k] = v / 4;
}

__global__ void qubo_finish_f64_kernel(double* F, int S, const double* off4)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    F[k] = (F[k] + *off4) * 0.25;
}

}  // namespace

cudaError_t launch_qubo_prep(const void* a, const void* b, int n, int dtype, void* Jout, void* hout, void* off4,
                             unsigned* flag, cudaStream_t s)
{
    if (dtype == 0)
        qubo_prep_kernel<int, int, long long><<<1, kQThreads, 0, s>>>(
            static_cast<const int*>(a), static_cast<const int*>(b), n, static_cast<int*>(Jout),
            static_cast<int*>(hout), static_cast<long long*>(off4), flag);
    else if (dtype == 1)
        qubo_prep_kernel<float, double, double><<<1, kQThreads, 0, s>>>(
            static_cast<const float*>(a), static_cast<const float*>(b), n, static_cast<double*>(Jout),
            static_cast<double*>(hout), static_cast<double*>(off4), flag);
    else
        qubo_prep_kernel<double, double, double><<<1, kQThreads, 0, s>>>(
            static_cast<const double*>(a), static_cast<const double*>(b), n, static_cast<double*>(Jout),
            static_cast<double*>(hout), static_cast<double*>(off4), flag);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_potts2_prep(const void* J, const void* h, int n, int dtype, void* Jout, void* hout, void* cst,
                               unsigned* flag, cudaStream_t s)
{
    if (dtype == 0)
        potts2_prep_kernel<int, int, long long><<<1, kQThreads, 0, s>>>(
            static_cast<const int*>(J), static_cast<const int*>(h), n, static_cast<int*>(Jout),
            static_cast<int*>(hout), static_cast<long long*>(cst), flag);
    else if (dtype == 1)
        potts2_prep_kernel<float, double, double><<<1, kQThreads, 0, s>>>(
            static_cast<const float*>(J), static_cast<const float*>(h), n, static_cast<double*>(Jout),
            static_cast<double*>(hout), static_cast<double*>(cst), flag);
    else
        potts2_prep_kernel<double, double, double><<<1, kQThreads, 0, s>>>(
            static_cast<const double*>(J), static_cast<const double*>(h), n, static_cast<double*>(Jout),
            static_cast<double*>(hout), static_cast<double*>(cst), flag);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_potts2_finish(void* E, int S, int dtype, const void* cst, unsigned* flag, cudaStream_t s,
                                 const unsigned* map_flag)
{
    const int blocks = (S + 255) / 256;
    if (dtype == 0)
        potts2_finish_i64_kernel<<<blocks, 256, 0, s>>>(static_cast<long long*>(E), S,
                                                        static_cast<const long long*>(cst), flag, map_flag);
    else
        potts2_finish_f64_kernel<<<blocks, 256, 0, s>>>(static_cast<double*>(E), S, static_cast<const double*>(cst));
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_qubo_finish(void* F, int S, int dtype, const void* off4, unsigned* flag, cudaStream_t s,
                               const unsigned* map_flag)
{
    const int blocks = (S + 255) / 256;
    if (dtype == 0)
        qubo_finish_i64_kernel<<<blocks, 256, 0, s>>>(static_cast<long long*>(F), S,
                                                      static_cast<const long long*>(off4), flag, map_flag);
    else
        qubo_finish_f64_kernel<<<blocks, 256, 0, s>>>(static_cast<double*>(F), S, static_cast<const double*>(off4));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
